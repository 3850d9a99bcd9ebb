// Per-length mixed-radix kernels: the runtime-radix pass of fftc_mixed.cuh with the line
// length, the tile height, the radix of every stage (and so every Ns, stride and loop
// bound) fixed at compile time. The stages, the shared-memory ping-pong and the HBM
// access patterns are those of k_mixed; what changes is that each stage's index
// arithmetic (the divisions of a butterfly index into line, group and twiddle index) and
// its radix dispatch disappear into constants, and the stage sequence is unrolled.
// Registered for the FP32 lengths that common workloads use (inst_mixed_ct.cu); any
// other length, or a plan whose tile differs, keeps the runtime-radix kernel.
#pragma once

#include <utility>

#include "fftc_mixed.cuh"

namespace fftc {

template <int... R>
struct MixedSched {
    static constexpr int S = sizeof...(R);
    __host__ __device__ static constexpr int radix(int s) {
        constexpr int r[] = {R...};
        return r[s];
    }
    __host__ __device__ static constexpr int ns(int s) {
        int p = 1;
        for (int i = 0; i < s; ++i) p *= radix(i);
        return p;
    }
    __host__ __device__ static constexpr int product() { return ns(S); }
};

// KIND / layouts as k_mixed; L points per line, C lines per tile, P the line pitch in shared
// memory (as the host sets it), R... the radices in stage order
template <int KIND, int LIN, int LOUT, int NT, int L, int C, int P, int... R>
struct MixedCt {
    using Sc = MixedSched<R...>;
    static constexpr int S = Sc::S;
    static_assert(Sc::product() == L, "the radices multiply to the line length");

    template <int s, int IO = 0, int LI = LAYOUT_IL, int LO = LAYOUT_IL, int K = KIND_ROWS, bool CF = false>
    __device__ __forceinline__ static void st(const MixedArgs &a, const float2 *src, float2 *dst, int64_t g0 = 0) {
        mixed_stage<Sc::radix(s), NT, float2, IO, LI, LO, K, CF, L, C, Sc::ns(s), P>(a, s, src, dst, g0);
    }

    // stages FIRST .. LAST-1 through shared memory; stage m reads the buffer stage m - 1 wrote
    // (stage FIRST - 1 wrote b0)
    template <int FIRST, int LAST, size_t... I>
    __device__ __forceinline__ static void mids(const MixedArgs &a, float2 *b0, float2 *b1, std::index_sequence<I...>) {
        ((st<FIRST + (int)I>(a, (I % 2 == 0) ? b0 : b1, (I % 2 == 0) ? b1 : b0), __syncthreads()), ...);
    }

    __device__ static void run(const MixedArgs &a) {
        extern __shared__ __align__(16) unsigned char sm_mixed_ct_raw[];
        float2 *buf0 = reinterpret_cast<float2 *>(sm_mixed_ct_raw);
        float2 *buf1 = buf0 + ((C * P + 1) & ~1);
        const int64_t g0 = (int64_t)blockIdx.x * C;
        // the split layout's short lines travel as flat 16-byte vectors per plane
        bool flat = false;
        if constexpr (KIND == KIND_ROWS && LIN == LAYOUT_SPLIT) flat = a.flat != 0 && !a.p.post_h;
        if (flat) {
            if constexpr (KIND == KIND_ROWS && LIN == LAYOUT_SPLIT) {
                rows_copy<LIN, NT, true>(a, g0, buf1);
                __syncthreads();
                st<0>(a, buf1, buf0);
                __syncthreads();
                mids<1, S>(a, buf0, buf1, std::make_index_sequence<S - 1>{});
                rows_copy<LOUT, NT, false>(a, g0, ((S - 1) % 2 == 0) ? buf0 : buf1);
            }
        } else if constexpr (S == 1) {
            constexpr bool CF = KIND == KIND_COLS;
            st<0, 3, LIN, LOUT, KIND, CF>(a, nullptr, nullptr, g0);
        } else if constexpr (KIND == KIND_ROWS) {
            {
                st<0, 1, LIN, LOUT>(a, nullptr, buf0, g0);
                __syncthreads();
                mids<1, S - 1>(a, buf0, buf1, std::make_index_sequence<S - 2>{});
                st<S - 1, 2, LIN, LOUT>(a, ((S - 2) % 2 == 0) ? buf0 : buf1, nullptr, g0);
            }
        } else {
            constexpr bool CF_IN = KIND == KIND_COLS;
            st<0, 1, LIN, LOUT, KIND, CF_IN>(a, nullptr, buf0, g0);
            __syncthreads();
            mids<1, S - 1>(a, buf0, buf1, std::make_index_sequence<S - 2>{});
            st<S - 1, 2, LIN, LOUT, KIND, true>(a, ((S - 2) % 2 == 0) ? buf0 : buf1, nullptr, g0);
        }
    }
};

template <int KIND, int LIN, int LOUT, int NT, int L, int C, int P, int... R>
__global__ void __launch_bounds__(NT) k_mixed_ct(const __grid_constant__ MixedArgs a) {
    MixedCt<KIND, LIN, LOUT, NT, L, C, P, R...>::run(a);
}

// registry entry: matched against a pass's kind, layouts, threads, L, C, pitch and radices
struct MixedCtEntry {
    int kind, lin, lout, nt, L, C, pitch, nst;
    int8_t radix[8];
    MixedKernel kernel;
};

template <int KIND, int LIN, int LOUT, int NT, int L, int C, int P, int... R>
constexpr MixedCtEntry mixed_ct_entry() {
    return MixedCtEntry{KIND, LIN, LOUT, NT, L, C, P, (int)sizeof...(R), {(int8_t)R...},
                        &k_mixed_ct<KIND, LIN, LOUT, NT, L, C, P, R...>};
}

// the compiled per-length kernel of this exact pass shape, or NULL (inst_mixed_ct.cu)
const MixedCtEntry *find_mixed_ct(int kind, int lin, int lout, int nt, int L, int C, int pitch, int nst,
                                  const int8_t *radix);

}  // namespace fftc
