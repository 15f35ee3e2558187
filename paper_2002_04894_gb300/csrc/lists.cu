// Connectivity (Eq. 2.2 and the inheritance rule of Sec. 2.1.1; the
// connectivity part of Algorithm 2): starting from the root's connection to
// itself, the children of every strongly connected pair of level l-1 are
// tested with the theta-criterion R + theta r <= theta d (R, r the larger and
// smaller radius, d the centre distance). Weak pairs become the M2L list of
// level l, strong pairs are refined further and at the leaf level form the
// P2P list. Both orientations of a pair are stored (the paper keeps only the
// lower triangle; the set of interactions is the same).
//
// GPU design: one thread per target box of level l walks its parent's strong
// list (ascending) and tests the two children of every source, so the output
// lists come out sorted per target with no sort. Count pass, exclusive scan,
// fill pass; the only host synchronisation per level is the total size.
// Degenerate pairs (theta = 0, or coincident centres) are always strong.

#include <algorithm>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

__device__ __forceinline__ bool theta_weak(double theta, const double *ca, double ra,
                                           const double *cb, double rb) {
    const double dx = __dsub_rn(ca[0], cb[0]);
    const double dy = __dsub_rn(ca[1], cb[1]);
    const double dz = __dsub_rn(ca[2], cb[2]);
    const double d = __dsqrt_rn(
        __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    const double R = ra > rb ? ra : rb;
    const double r = ra > rb ? rb : ra;
    return theta > 0.0 && d > 0.0 && __dadd_rn(R, __dmul_rn(theta, r)) <= __dmul_rn(theta, d);
}

template <bool kFill>
__global__ void k_lists(int level, double theta, const int32_t *__restrict__ pptr,
                        const int32_t *__restrict__ psrc, const double *__restrict__ centre,
                        const double *__restrict__ radius, int32_t *wcnt, int32_t *scnt,
                        const int32_t *__restrict__ wptr, const int32_t *__restrict__ sptr,
                        int32_t *wsrc, int32_t *ssrc) {
    const int64_t nt = (int64_t)1 << level;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int64_t off = nt - 1;
    const int64_t gt = off + t;
    const double ct[3] = {centre[3 * gt], centre[3 * gt + 1], centre[3 * gt + 2]};
    const double rt = radius[gt];
    const int64_t T = t >> 1;
    int32_t nw = 0, ns = 0;
    int32_t iw = kFill ? wptr[t] : 0, is = kFill ? sptr[t] : 0;
    for (int32_t e = pptr[T]; e < pptr[T + 1]; e++) {
        const int32_t S = psrc[e];
        for (int c = 0; c < 2; c++) {
            const int32_t s = 2 * S + c;
            const int64_t gs = off + s;
            const bool weak = theta_weak(theta, ct, rt, centre + 3 * gs, radius[gs]);
            if (kFill) {
                if (weak)
                    wsrc[iw++] = s;
                else
                    ssrc[is++] = s;
            } else {
                nw += weak;
                ns += !weak;
            }
        }
    }
    if (!kFill) {
        wcnt[t] = nw;
        scnt[t] = ns;
    }
}

// ---- exclusive scan of int32 counts: out[0..n], out[n] = total -------------
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ int32_t block_exclusive(int32_t v, int32_t *total) {
    __shared__ int32_t ws[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) ws[w] = incl;
    __syncthreads();
    if (w == 0) {
        int32_t x = lane < kScanThreads / 32 ? ws[lane] : 0;
        int32_t xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t t = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += t;
        }
        if (lane < kScanThreads / 32) ws[lane] = xi - x;
        if (lane == 31) *total = xi;
    }
    __syncthreads();
    const int32_t r = ws[w] + incl - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_tiles(const int32_t *in, int32_t *out, int64_t n, int32_t *tile_sums) {
    __shared__ int32_t tot;
    const int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanItems;
    int32_t v[kScanItems], s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        v[j] = base + j < n ? in[base + j] : 0;
        s += v[j];
    }
    int32_t run = block_exclusive(s, &tot);
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_sums(int32_t *tile_sums, int64_t ntiles, int32_t *total_out) {
    // single block; ntiles <= kScanTile
    __shared__ int32_t tot;
    const int64_t base = threadIdx.x * (int64_t)kScanItems;
    int32_t v[kScanItems], s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        v[j] = base + j < ntiles ? tile_sums[base + j] : 0;
        s += v[j];
    }
    int32_t run = block_exclusive(s, &tot);
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        if (base + j < ntiles) tile_sums[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == 0) *total_out = tot;
}

__global__ void k_scan_add(int32_t *out, int64_t n, const int32_t *tile_sums) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_sums[i / kScanTile];
}

// sum over strong leaf pairs (t, s) of n_t * n_s
__global__ void k_p2p_work(int B, const int32_t *sptr, const int32_t *ssrc, const int32_t *count,
                           unsigned long long *acc) {
    const int64_t nt = (int64_t)1 << B;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (t < nt) {
        const int64_t off = nt - 1;
        unsigned long long ns = 0;
        for (int32_t e = sptr[t]; e < sptr[t + 1]; e++) ns += (unsigned long long)count[off + ssrc[e]];
        v = ns * (unsigned long long)count[off + t];
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(acc, v);
}

}  // namespace

cudaError_t scan_exclusive(Plan &P, const int32_t *in, int32_t *out, int64_t n) {
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles > kScanTile) return cudaErrorInvalidValue;
    int32_t *sums = (int32_t *)dalloc(P, (size_t)std::max<int64_t>(ntiles, 1) * 4);
    if (!sums) return cudaErrorMemoryAllocation;
    if (n > 0) {
        FMM_LAUNCH(k_scan_tiles, (unsigned)ntiles, kScanThreads, 0, P.stream, in, out, n, sums);
        FMM_LAUNCH(k_scan_sums, 1, kScanThreads, 0, P.stream, sums, ntiles, out + n);
        if (ntiles > 1)
            FMM_LAUNCH(k_scan_add, (unsigned)((n + 255) / 256), 256, 0, P.stream, out, n, sums);
    } else {
        cudaMemsetAsync(out, 0, 4, P.stream);
    }
    dfree(P, sums, (size_t)std::max<int64_t>(ntiles, 1) * 4);
    return cudaGetLastError();
}

cudaError_t lists_build(Plan &P) {
    cudaStream_t st = P.stream;
    // level 0: the root is strongly connected to itself
    P.wptr[0] = (int32_t *)palloc(P, 8);
    P.sptr[0] = (int32_t *)palloc(P, 8);
    P.ssrc[0] = (int32_t *)palloc(P, 4);
    P.wsrc[0] = nullptr;
    if (!P.wptr[0] || !P.sptr[0] || !P.ssrc[0]) return cudaErrorMemoryAllocation;
    const int32_t w0[2] = {0, 0}, s0[2] = {0, 1}, src0 = 0;
    cudaMemcpyAsync(P.wptr[0], w0, 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(P.sptr[0], s0, 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(P.ssrc[0], &src0, 4, cudaMemcpyHostToDevice, st);
    P.nweak[0] = 0;
    P.nstrong[0] = 1;
    int32_t *totals = nullptr;
    cudaMallocHost(&totals, 8);
    for (int l = 1; l <= P.B; l++) {
        const int64_t nt = (int64_t)1 << l;
        // every child pair of a strong parent pair is a candidate: 4 per parent pair
        if (4 * P.nstrong[l - 1] > 0x7fffffffLL) {
            P.capacity_exceeded = true;
            cudaFreeHost(totals);
            return cudaSuccess;
        }
        int32_t *wcnt = (int32_t *)dalloc(P, nt * 4), *scnt = (int32_t *)dalloc(P, nt * 4);
        P.wptr[l] = (int32_t *)palloc(P, (nt + 1) * 4);
        P.sptr[l] = (int32_t *)palloc(P, (nt + 1) * 4);
        if (!wcnt || !scnt || !P.wptr[l] || !P.sptr[l]) return cudaErrorMemoryAllocation;
        const unsigned grid = (unsigned)((nt + 127) / 128);
        FMM_LAUNCH(k_lists<false>, grid, 128, 0, st, l, P.theta, P.sptr[l - 1], P.ssrc[l - 1], P.centre,
                                             P.radius, wcnt, scnt, nullptr, nullptr, nullptr,
                                             nullptr);
        cudaError_t e = scan_exclusive(P, wcnt, P.wptr[l], nt);
        if (e == cudaSuccess) e = scan_exclusive(P, scnt, P.sptr[l], nt);
        if (e != cudaSuccess) return e;
        cudaMemcpyAsync(totals, P.wptr[l] + nt, 4, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(totals + 1, P.sptr[l] + nt, 4, cudaMemcpyDeviceToHost, st);
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        P.nweak[l] = totals[0];
        P.nstrong[l] = totals[1];
        P.wsrc[l] = (int32_t *)palloc(P, (size_t)std::max<int64_t>(P.nweak[l], 1) * 4);
        P.ssrc[l] = (int32_t *)palloc(P, (size_t)std::max<int64_t>(P.nstrong[l], 1) * 4);
        if (!P.wsrc[l] || !P.ssrc[l]) return cudaErrorMemoryAllocation;
        FMM_LAUNCH(k_lists<true>, grid, 128, 0, st, l, P.theta, P.sptr[l - 1], P.ssrc[l - 1], P.centre,
                                            P.radius, nullptr, nullptr, P.wptr[l], P.sptr[l],
                                            P.wsrc[l], P.ssrc[l]);
        dfree(P, wcnt, nt * 4);
        dfree(P, scnt, nt * 4);
    }
    // exact P2P work (sum of n_t * n_s over strong leaf pairs)
    unsigned long long *acc = (unsigned long long *)dalloc(P, 8);
    if (!acc) return cudaErrorMemoryAllocation;
    cudaMemsetAsync(acc, 0, 8, st);
    const int64_t nl = (int64_t)1 << P.B;
    FMM_LAUNCH(k_p2p_work, (unsigned)((nl + 255) / 256), 256, 0, st, P.B, P.sptr[P.B], P.ssrc[P.B], P.count,
                                                           acc);
    unsigned long long h = 0;
    cudaMemcpyAsync(&h, acc, 8, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    P.p2p_interactions = (int64_t)h;
    dfree(P, acc, 8);
    cudaFreeHost(totals);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace fmm
