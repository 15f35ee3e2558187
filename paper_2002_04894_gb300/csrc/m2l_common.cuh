// Pieces shared by the M2L kernels: the flattened table of weak pairs over
// all levels, the lookup of a pair's boxes, and the segmented warp sum of the
// contributions to equal targets (the pair list is sorted by target).
#pragma once

#include "fmm_internal.cuh"

namespace fmm {

__device__ __forceinline__ void pair_of(const PairTable &PT, int64_t g, int64_t &gt, int64_t &gs) {
    int l = PT.lmin;
    while (l < PT.lmax && g >= PT.off[l + 1]) l++;
    const int64_t e = g - PT.off[l];
    const int64_t boff = ((int64_t)1 << l) - 1;
    gt = boff + PT.tgt[l][e];
    gs = boff + PT.src[l][e];
}

// Segmented sum over lanes of equal target (the pair list is sorted by
// target): after the five steps the first lane of each run holds the run's
// sum. same[j] says whether lane + 2^j belongs to this lane's run.
template <typename R>
__device__ __forceinline__ R seg_sum(R v, const bool (&same)[5]) {
#pragma unroll
    for (int j = 0; j < 5; j++) {
        const R o = __shfl_down_sync(0xffffffffu, v, 1 << j);
        if (same[j]) v += o;
    }
    return v;
}

__device__ __forceinline__ void seg_setup(int64_t tgt, bool (&same)[5], bool &head) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < 5; j++) {
        const int64_t o = __shfl_down_sync(0xffffffffu, tgt, 1 << j);
        same[j] = (lane + (1 << j) < 32) && o == tgt;
    }
    const int64_t up = __shfl_up_sync(0xffffffffu, tgt, 1);
    head = tgt >= 0 && (lane == 0 || up != tgt);
}

PairTable pair_table(const Plan &P);
int64_t total_weak(const Plan &P);
long double factl(int n);
long double wigner_half_pi(int n, int k, int m);  // d^n_{km}(pi/2)

}  // namespace fmm
