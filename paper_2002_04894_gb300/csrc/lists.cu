// Connectivity (Eq. 2.2 and the inheritance rule of Sec. 2.1.1; the
// connectivity part of Algorithm 2): starting from the root's connection to
// itself, the children of every strongly connected pair of level l-1 (or of
// level l-step for levels of 2^step children, step = 3 being the octree) are
// tested with the theta-criterion R + theta r <= theta d (R, r the larger and
// smaller radius, d the centre distance). Weak pairs become the M2L list of
// level l, strong pairs are refined further and at the leaf level form the
// P2P list. Both orientations of a pair are stored (the paper keeps only the
// lower triangle; the set of interactions is the same).
//
// GPU design: the work is flattened over the parent level's strong pairs, not
// over target boxes: clustered point sets make some boxes (large, sparse
// ones) strongly connected to a large share of their level, and a
// thread-per-target loop would run as long as the longest list. One thread
// per parent pair tests its four child pairs and writes the flags in
// target-major, source-ascending order; one scan of the weak flags gives the
// CSR slot of every weak and strong pair. The only host synchronisation per
// level is the total size.
// Degenerate pairs (theta = 0, or coincident centres) are always strong.

#include <algorithm>
#include <vector>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

__device__ __forceinline__ bool theta_weak(double theta, const double *ca, double ra,
                                           const double *cb, double rb) {
    const double dx = __dsub_rn(ca[0], cb[0]);
    const double dy = __dsub_rn(ca[1], cb[1]);
    const double dz = __dsub_rn(ca[2], cb[2]);
    const double s = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double R = ra > rb ? ra : rb;
    const double r = ra > rb ? rb : ra;
    if (!(theta > 0.0) || !(s > 0.0)) return false;
    const double L = __dadd_rn(R, __dmul_rn(theta, r));
    // decided on squares when clearly away from the boundary (the rounding of
    // the sqrt form is ~2u, the margin 1e-12); the exact test otherwise, so
    // the outcome is that of L <= theta * sqrt(s) in every case
    const double a = L * L, b = theta * theta * s;
    if (a < b * (1.0 - 1e-12)) return true;
    if (a > b * (1.0 + 1e-12)) return false;
    return L <= __dmul_rn(theta, __dsqrt_rn(s));
}

// One thread per strongly connected pair (T, S) of the parent level: its
// C x C child pairs (C T + a, C S + b), C = 2^step children per box (step
// bisections per level; 3 for octree levels), are tested and their flags
// written at their position in the target-major candidate order
//   cpos = C^2 sptr[T] + a * C len(T) + C (e - sptr[T]) + b,
// i.e. grouped by target C T + a and, inside a target, by ascending source
// (the parent's sources are ascending). A scan of the weak flags then places
// every weak and strong pair directly in its sorted CSR slot.
__global__ void k_cand(int level, int step, int64_t npar, double theta, const int32_t *__restrict__ pptr,
                       const int32_t *__restrict__ psrc, const int32_t *__restrict__ prow,
                       const double *__restrict__ centre, const double *__restrict__ radius,
                       int32_t *__restrict__ flag, int32_t *__restrict__ csrc,
                       int32_t *__restrict__ ctgt) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= npar) return;
    const int C = 1 << step;
    const int32_t T = prow[e], S = psrc[e];
    const int32_t b0 = pptr[T], len = pptr[T + 1] - b0;
    const int64_t off = ((int64_t)1 << level) - 1;
    for (int a = 0; a < C; a++) {
        const int32_t t = C * T + a;
        const int64_t gt = off + t;
        const int64_t base = (int64_t)C * C * b0 + (int64_t)a * C * len + (int64_t)C * (e - b0);
        for (int b = 0; b < C; b++) {
            const int32_t s = C * S + b;
            const int64_t gs = off + s;
            flag[base + b] = theta_weak(theta, centre + 3 * gt, radius[gt], centre + 3 * gs, radius[gs]);
            csrc[base + b] = s;
            ctgt[base + b] = t;
        }
    }
}

__global__ void k_cand_scatter(int64_t ncand, const int32_t *__restrict__ flag,
                               const int32_t *__restrict__ wpos, const int32_t *__restrict__ csrc,
                               const int32_t *__restrict__ ctgt, int32_t *__restrict__ wsrc,
                               int32_t *__restrict__ wrow, int32_t *__restrict__ ssrc,
                               int32_t *__restrict__ srow) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= ncand) return;
    const int32_t w = wpos[c];
    if (flag[c]) {
        wsrc[w] = csrc[c];
        wrow[w] = ctgt[c];
    } else {
        const int64_t sp = c - w;
        ssrc[sp] = csrc[c];
        srow[sp] = ctgt[c];
    }
}

// CSR row pointers of level `level` from the parent level's: target
// t = C T + a starts at candidate C^2 sptr[T] + a * C len(T).
__global__ void k_cand_ptrs(int level, int step, const int32_t *__restrict__ pptr,
                            const int32_t *__restrict__ wpos, int64_t ncand,
                            int32_t *__restrict__ wptr, int32_t *__restrict__ sptr) {
    const int64_t nt = (int64_t)1 << level;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t > nt) return;
    const int64_t C = (int64_t)1 << step;
    int64_t first;
    if (t == nt) {
        first = ncand;
    } else {
        const int64_t T = t >> step, a = t & (C - 1);
        first = C * C * pptr[T] + a * C * (pptr[T + 1] - pptr[T]);
    }
    const int32_t w = wpos[first];
    wptr[t] = w;
    sptr[t] = (int32_t)(first - w);
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

// per target leaf the near source points (sum of n_s over its strong leaf
// pairs), and in total the sum over strong leaf pairs (t, s) of n_t * n_s
__global__ void k_p2p_work(int B, const int32_t *sptr, const int32_t *ssrc, const int32_t *count,
                           unsigned long long *acc, long long *per_leaf) {
    const int64_t nt = (int64_t)1 << B;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (t < nt) {
        const int64_t off = nt - 1;
        unsigned long long ns = 0;
        for (int32_t e = sptr[t]; e < sptr[t + 1]; e++) ns += (unsigned long long)count[off + ssrc[e]];
        v = ns * (unsigned long long)count[off + t];
        per_leaf[t] = (long long)ns;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(acc, v);
}

}  // namespace

cudaError_t scan_exclusive(Plan &P, const int32_t *in, int32_t *out, int64_t n) {
    if (n <= 0) {
        cudaMemsetAsync(out, 0, 4, P.stream);
        return cudaGetLastError();
    }
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles == 1) {
        int32_t *sums = (int32_t *)dalloc(P, 4);
        if (!sums) return cudaErrorMemoryAllocation;
        FMM_LAUNCH(k_scan_tiles, 1, kScanThreads, 0, P.stream, in, out, n, sums);
        FMM_LAUNCH(k_scan_sums, 1, kScanThreads, 0, P.stream, sums, 1, out + n);
        return cudaGetLastError();
    }
    // tile sums -> their exclusive scan (recursively) -> add back
    int32_t *sums = (int32_t *)dalloc(P, (size_t)ntiles * 4);
    int32_t *sscan = (int32_t *)dalloc(P, (size_t)(ntiles + 1) * 4);
    if (!sums || !sscan) return cudaErrorMemoryAllocation;
    FMM_LAUNCH(k_scan_tiles, (unsigned)ntiles, kScanThreads, 0, P.stream, in, out, n, sums);
    cudaError_t e = scan_exclusive(P, sums, sscan, ntiles);
    if (e != cudaSuccess) return e;
    FMM_LAUNCH(k_scan_add, (unsigned)((n + 255) / 256), 256, 0, P.stream, out, n, sscan);
    cudaMemcpyAsync(out + n, sscan + ntiles, 4, cudaMemcpyDeviceToDevice, P.stream);
    return cudaGetLastError();
}

cudaError_t lists_build(Plan &P) {
    cudaStream_t st = P.stream;
    // level 0: the root is strongly connected to itself
    P.wptr[0] = (int32_t *)palloc(P, 8);
    P.sptr[0] = (int32_t *)palloc(P, 8);
    P.ssrc[0] = (int32_t *)palloc(P, 4);
    P.wsrc[0] = nullptr;
    P.wrow[0] = nullptr;
    int32_t *srow_prev = (int32_t *)dalloc(P, 4);
    if (!P.wptr[0] || !P.sptr[0] || !P.ssrc[0] || !srow_prev) return cudaErrorMemoryAllocation;
    const int32_t w0[2] = {0, 0}, s0[2] = {0, 1}, zero = 0;
    cudaMemcpyAsync(P.wptr[0], w0, 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(P.sptr[0], s0, 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(P.ssrc[0], &zero, 4, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(srow_prev, &zero, 4, cudaMemcpyHostToDevice, st);
    P.nweak[0] = 0;
    P.nstrong[0] = 1;
    int32_t totals[2] = {0, 0};  // level sizes, read back synchronously
    cudaError_t e = cudaSuccess;
    const int step = P.step, C = 1 << step;
    for (int l = 1; l <= P.B; l++) {
        const int64_t nt = (int64_t)1 << l;
        if (l % step) {
            // a bisection level inside a level of 2^step children: no pairs
            P.wptr[l] = (int32_t *)palloc(P, (nt + 1) * 4);
            P.sptr[l] = (int32_t *)palloc(P, (nt + 1) * 4);
            P.wsrc[l] = (int32_t *)palloc(P, 4);
            P.wrow[l] = (int32_t *)palloc(P, 4);
            P.ssrc[l] = (int32_t *)palloc(P, 4);
            if (!P.wptr[l] || !P.sptr[l] || !P.wsrc[l] || !P.wrow[l] || !P.ssrc[l]) return cudaErrorMemoryAllocation;
            cudaMemsetAsync(P.wptr[l], 0, (nt + 1) * 4, st);
            cudaMemsetAsync(P.sptr[l], 0, (nt + 1) * 4, st);
            P.nweak[l] = 0;
            P.nstrong[l] = 0;
            continue;
        }
        const int lp = l - step;
        const int64_t npar = P.nstrong[lp], ncand = (int64_t)C * C * npar;
        if (ncand > 0x7fffffffLL) {
            P.capacity_exceeded = true;
            return cudaSuccess;
        }
        int32_t *flag = (int32_t *)dalloc(P, (size_t)ncand * 4);
        int32_t *wpos = (int32_t *)dalloc(P, (size_t)(ncand + 1) * 4);
        int32_t *csrc = (int32_t *)dalloc(P, (size_t)ncand * 4);
        int32_t *ctgt = (int32_t *)dalloc(P, (size_t)ncand * 4);
        P.wptr[l] = (int32_t *)palloc(P, (nt + 1) * 4);
        P.sptr[l] = (int32_t *)palloc(P, (nt + 1) * 4);
        if (!flag || !wpos || !csrc || !ctgt || !P.wptr[l] || !P.sptr[l]) return cudaErrorMemoryAllocation;
        FMM_LAUNCH(k_cand, (unsigned)((npar + 127) / 128), 128, 0, st, l, step, npar, P.theta, P.sptr[lp],
                   P.ssrc[lp], srow_prev, P.centre, P.radius, flag, csrc, ctgt);
        e = scan_exclusive(P, flag, wpos, ncand);
        if (e != cudaSuccess) return e;
        FMM_LAUNCH(k_cand_ptrs, (unsigned)((nt + 1 + 255) / 256), 256, 0, st, l, step, P.sptr[lp], wpos,
                   ncand, P.wptr[l], P.sptr[l]);
        cudaMemcpyAsync(totals, wpos + ncand, 4, cudaMemcpyDeviceToHost, st);
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        P.nweak[l] = totals[0];
        P.nstrong[l] = ncand - totals[0];
        P.wsrc[l] = (int32_t *)palloc(P, (size_t)std::max<int64_t>(P.nweak[l], 1) * 4);
        P.wrow[l] = (int32_t *)palloc(P, (size_t)std::max<int64_t>(P.nweak[l], 1) * 4);
        P.ssrc[l] = (int32_t *)palloc(P, (size_t)std::max<int64_t>(P.nstrong[l], 1) * 4);
        int32_t *srow = (int32_t *)dalloc(P, (size_t)std::max<int64_t>(P.nstrong[l], 1) * 4);
        if (!P.wsrc[l] || !P.wrow[l] || !P.ssrc[l] || !srow) return cudaErrorMemoryAllocation;
        FMM_LAUNCH(k_cand_scatter, (unsigned)((ncand + 255) / 256), 256, 0, st, ncand, flag, wpos, csrc,
                   ctgt, P.wsrc[l], P.wrow[l], P.ssrc[l], srow);
        srow_prev = srow;
    }
    // exact P2P work (sum of n_t * n_s over strong leaf pairs). The near
    // field runs as work units of up to kP2PTile targets of one leaf, so that
    // a few large leaves still fill the GPU; units go heaviest first, so that
    // the long ones start early instead of forming the tail of the launch.
    const int64_t nl = (int64_t)1 << P.B;
    unsigned long long *acc = (unsigned long long *)dalloc(P, 8);
    long long *nsrc = (long long *)dalloc(P, (size_t)nl * 8);
    if (!acc || !nsrc) return cudaErrorMemoryAllocation;
    cudaMemsetAsync(acc, 0, 8, st);
    FMM_LAUNCH(k_p2p_work, (unsigned)((nl + 255) / 256), 256, 0, st, P.B, P.sptr[P.B], P.ssrc[P.B],
               P.count, acc, nsrc);
    std::vector<long long> hns((size_t)nl);
    std::vector<int32_t> hcnt((size_t)nl);
    unsigned long long h = 0;
    cudaMemcpyAsync(&h, acc, 8, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hns.data(), nsrc, (size_t)nl * 8, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hcnt.data(), P.count + (nl - 1), (size_t)nl * 4, cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    P.p2p_interactions = (int64_t)h;
    if (e != cudaSuccess) return e;
    std::vector<int2> units;
    std::vector<long long> uw;
    units.reserve((size_t)nl);
    uw.reserve((size_t)nl);
    for (int64_t t = 0; t < nl; t++)
        for (int32_t tb = 0; tb < hcnt[t]; tb += kP2PTile) {
            units.push_back(make_int2((int)t, tb));
            uw.push_back((long long)std::min(kP2PTile, hcnt[t] - tb) * hns[t]);
        }
    std::vector<int32_t> idx(units.size());
    for (size_t i = 0; i < idx.size(); i++) idx[i] = (int32_t)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return uw[a] > uw[b]; });
    std::vector<int2> sorted(units.size());
    for (size_t i = 0; i < idx.size(); i++) sorted[i] = units[idx[i]];
    P.p2p_nunits = (int64_t)sorted.size();
    P.p2p_units = (int2 *)palloc(P, std::max<size_t>(sorted.size(), 1) * sizeof(int2));
    if (!P.p2p_units) return cudaErrorMemoryAllocation;
    if (!sorted.empty())
        e = cudaMemcpyAsync(P.p2p_units, sorted.data(), sorted.size() * sizeof(int2),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace fmm
