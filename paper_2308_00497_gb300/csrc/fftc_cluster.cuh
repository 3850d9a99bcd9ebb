// Single-pass transforms of n = 2^15 .. 2^18 points on a thread-block cluster: Eq. 1 once
// more at the cluster level, n = n1 n2, with the middle permutation (the stride
// permutation of Eq. 1 between its two factors) carried by distributed shared memory
// instead of an HBM workspace, so every element crosses HBM once (read once, written once).
//
// A cluster of R CTAs owns one transform at a time (persistent over the batch); CTA r holds
// Q = n / R elements in one shared-memory buffer:
//   phase A  columns j2 in [r n2/R, (r+1) n2/R): n2/R column FFTs of length n1 at element
//            stride n2 (Table 1's I (x) DFT on the stride-permuted input), loaded as one
//            tensor-map box per 256 rows into the buffer; the exchanges between radix stages
//            reuse the buffer; the last stage multiplies by the diagonal w_n^(j2 k1) and
//            writes output k1 of column j2 into row k1 mod (n1/R), position j2, of the buffer
//            of CTA k1 / (n1/R) (st.shared::cluster), after a cluster barrier that ends every
//            CTA's reads of its own buffer;
//   phase B  after a second cluster barrier, rows k1 in [r n1/R, (r+1) n1/R): n1/R row FFTs
//            of length n2 straight from the buffer, stored to HBM at k1 + n1 k2 (coalesced
//            runs of n1/R elements).
// The buffer is refilled with the next transform's columns as soon as phase B's last
// shared-memory read is done, so the HBM reads of transform t + 1 overlap the end of t.
// Every CTA of a cluster runs the same sequence of cluster barriers, whatever happens: a
// landing wait that runs out sets the plan's error word and the CTA goes on (with
// undefined data) rather than leaving the cluster's barriers unbalanced.
#pragma once

#include "fftc_pipe.cuh"

namespace fftc {

// (a kernel parameter: the tensor maps must stay in parameter space for the bulk copies)
struct ClusterArgs {
    PipeArgs feed;  // phase A (KIND_CLUSTER_A, landed columns) and its input tensor maps
    PassParams b;   // phase B (KIND_ROWST, landed rows)
    int64_t batch;
};

// the cluster barrier as a tile hook: every thread of the cluster, after the last local read
struct ClusterBarrierHook {
    static constexpr bool active = true;
    __device__ __forceinline__ void operator()() const { cluster_sync_all(); }
};

template <class PA, class PB, int R>
struct ClusterPass {
    static_assert(PA::NT == PB::NT, "both phases run in the same CTA");
    static_assert(PA::C_LINES * PA::L == PB::C_LINES * PB::L, "both phases hold the CTA's Q elements");
    static_assert(PA::C_LINES * R == PB::L && PB::C_LINES * R == PA::L, "n = n1 n2 split over R CTAs");
    static constexpr int NT = PA::NT;
    static constexpr int Q = PA::C_LINES * PA::L;
    static constexpr int WA = PA::C_LINES * PA::PITCH, WB = PB::C_LINES * PB::PITCH;
    static constexpr int WORDS = ((Q > WA ? (Q > WB ? Q : WB) : (WA > WB ? WA : WB)) + 15) / 16 * 16;
    static constexpr int SMEM = WORDS * (int)sizeof(float2) + 128;
    using Feed = PipeTile<PA, 1, true>;  // the tensor-map column loads of a four-step pass 1

    struct Refill {
        static constexpr bool active = true;
        const PipeArgs *pa;
        int64_t tile;
        float2 *buf;
        uint64_t *bar;
        __device__ __forceinline__ void operator()() const {
            if (tile >= 0 && threadIdx.x == 0) {
                fence_proxy_async_smem();
                Feed::issue(*pa, tile, buf, bar);
            }
        }
    };

    __device__ static void run(const ClusterArgs &args) {
        const PipeArgs &feed = args.feed;
        const PassParams &pa = feed.p;
        float2 *buf = reinterpret_cast<float2 *>(dyn_smem_base128());
        __shared__ __align__(8) uint64_t bar;
        const uint32_t rank = cluster_ctarank();
        const int64_t cid = blockIdx.x / R, ncl = gridDim.x / R;
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (threadIdx.x == 0 && cid < args.batch) Feed::issue(feed, cid * R + rank, buf, &bar);
        const long long limit = pa.spin_limit > 0 ? (long long)pa.spin_limit : kMbarSpinLimit;
        bool pending = false;  // a copy whose wait ran out may still be in flight
        uint32_t k = 0;
        for (int64_t t = cid; t < args.batch; t += ncl, ++k) {
            if (!mbar_wait_bounded(&bar, k & 1u, limit)) {
                if (threadIdx.x == 0 && pa.err) atomicExch(pa.err, 4);
                pending = true;
            }
            PA::run_tile_landed(pa, t * R + rank, buf, ClusterBarrierHook());
            cluster_sync_all();  // every CTA's phase-A results are in its peers' buffers
            const int64_t next = t + ncl;
            PB::run_tile_landed(args.b, t * R + rank, buf,
                                Refill{&feed, next < args.batch ? next * R + rank : -1, buf, &bar});
        }
        if (pending) mbar_wait_bounded(&bar, k & 1u, limit);
        cluster_sync_all();  // no CTA leaves while a peer may still address its shared memory
    }
};

template <class PA, class PB, int R>
__global__ void __launch_bounds__(PA::NT, (1024 / PA::NT) > 0 ? (1024 / PA::NT) : 1)
    k_cluster(const __grid_constant__ ClusterArgs args) {
    ClusterPass<PA, PB, R>::run(args);
}

template <class PA, class PB, int R>
struct ClusterLauncher {
    using CP = ClusterPass<PA, PB, R>;
    static int &clusters() {
        static int c = 0;
        return c;
    }
    static cudaError_t prepare() {
        auto kern = k_cluster<PA, PB, R>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, CP::SMEM);
        if (e != cudaSuccess) return e;
        if (R > 8 && (e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
            return e;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = R;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(R, 1, 1);
        cfg.blockDim = dim3(CP::NT, 1, 1);
        cfg.dynamicSmemBytes = CP::SMEM;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if ((e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg)) != cudaSuccess) return e;
        if (n <= 0) return cudaErrorInvalidConfiguration;
        clusters() = n;
        return cudaSuccess;
    }
    static cudaError_t launch(const PassParams &a, const PassParams &b, int64_t batch, cudaStream_t st) {
        if (batch <= 0) return cudaSuccess;
        if (clusters() == 0) {
            cudaError_t e = prepare();
            if (e != cudaSuccess) return e;
        }
        ClusterArgs args;
        memset(&args, 0, sizeof(args));
        args.feed.p = a;
        args.b = b;
        args.batch = batch;
        if (!encode_cols_maps(a, PA::L == 0 ? 0 : __builtin_ctz(PA::L), PA::C_LINES, PA::LIN_LAYOUT, args.feed.tm))
            return cudaErrorInvalidValue;
        const int64_t ncl = batch < clusters() ? batch : clusters();
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = R;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(ncl * R), 1, 1);
        cfg.blockDim = dim3(CP::NT, 1, 1);
        cfg.dynamicSmemBytes = CP::SMEM;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_cluster<PA, PB, R>, args);
    }
};

// registry entry: n = 2^(LOG1 + LOG2), phase A columns of n1 = 2^LOG1, phase B rows of
// n2 = 2^LOG2, R CTAs per transform, 2^LOGE elements per thread, one layout in and out
template <int LOG1, int LOG2, int R, int LOGE, int LAY>
constexpr ClusterEntry cluster_entry() {
    using PA = Pass<LOG1, LOGE, (1 << LOG2) / R, KIND_CLUSTER_A, LAY, LAYOUT_IL, false, LOG2>;
    using PB = Pass<LOG2, LOGE, (1 << LOG1) / R, KIND_ROWST, LAYOUT_IL, LAY, false, LOG1>;
    using L = ClusterLauncher<PA, PB, R>;
    return ClusterEntry{LOG1 + LOG2, LOG1, LOGE, R, LAY, PA::NT, ClusterPass<PA, PB, R>::SMEM, &L::launch, &L::prepare};
}

}  // namespace fftc
