// Instantiations of the cluster single pass (fftc_cluster.cuh): n = 2^15 .. 2^18 as
// n1 x n2 over clusters of R CTAs holding Q = n / R elements each, 16 elements per thread:
//   Q = 2^13 (512 threads, ~68 KB, two or three CTAs per SM): 2^15 (R 4), 2^16 (R 8), 2^17 (R 16);
//   Q = 2^14 (1024 threads, ~135 KB, one CTA per SM):          2^15 (R 2), 2^16 (R 4), 2^17 (R 8),
//                                                               2^18 (R 16).
#include "fftc_cluster.cuh"

namespace fftc {

#define CL2(LOG1, LOG2, R) cluster_entry<LOG1, LOG2, R, 4, LAYOUT_IL>(), cluster_entry<LOG1, LOG2, R, 4, LAYOUT_SPLIT>()

static const ClusterEntry kClusterTable[] = {
    CL2(7, 8, 4), CL2(8, 8, 8), CL2(8, 9, 16),
    CL2(7, 8, 2), CL2(8, 8, 4), CL2(8, 9, 8), CL2(9, 9, 16),
};

int cluster_kernel_count() { return (int)(sizeof(kClusterTable) / sizeof(kClusterTable[0])); }
const ClusterEntry *cluster_kernel_at(int i) {
    return (i >= 0 && i < cluster_kernel_count()) ? &kClusterTable[i] : nullptr;
}

}  // namespace fftc
