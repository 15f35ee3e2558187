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
    const double R = ra > rb ? ra : rb;
    const double r = ra > rb ? rb : ra;
    if (!(theta > 0.0)) return false;
    {
        // most candidates are far from the boundary: decided in single
        // precision (relative error ~1e-6 of L^2 / (theta^2 s)) with a 1e-4
        // margin, which cannot change the outcome; the rest, and any value
        // out of the comfortable float range, go to the double-precision test
        const float fx = (float)dx, fy = (float)dy, fz = (float)dz, ft = (float)theta;
        const float fs = fx * fx + fy * fy + fz * fz;
        const float fl = (float)R + ft * (float)r;
        const float fa = fl * fl, fb = ft * ft * fs;
        if (fs > 1e-30f && fs < 1e30f && fa > 1e-30f && fa < 1e30f && fb > 1e-30f && fb < 1e30f) {
            if (fa < fb * (1.0f - 1e-4f)) return true;
            if (fa > fb * (1.0f + 1e-4f)) return false;
        }
    }
    const double s = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (!(s > 0.0)) return false;
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
// The pre-test of theta_weak from the boxes' split float centres and float
// radii (no double arithmetic: GB300's FP64 pipe is narrow); 1 weak, 0
// strong, -1 undecided (near the boundary, or out of the comfortable float
// range): the double-precision test then decides.
__device__ __forceinline__ int theta_pretest(float ft, const float4 &ah, const float4 &al, const float4 &bh,
                                             const float4 &bl) {
    const float fx = offset_f(ah.x, bh.x, al.x, bl.x);
    const float fy = offset_f(ah.y, bh.y, al.y, bl.y);
    const float fz = offset_f(ah.z, bh.z, al.z, bl.z);
    const float R = fmaxf(ah.w, bh.w), r = fminf(ah.w, bh.w);
    const float fs = fx * fx + fy * fy + fz * fz;
    const float fl = R + ft * r;
    const float fa = fl * fl, fb = ft * ft * fs;
    if (fs > 1e-30f && fs < 1e30f && fa > 1e-30f && fa < 1e30f && fb > 1e-30f && fb < 1e30f) {
        if (fa < fb * (1.0f - 1e-4f)) return 1;
        if (fa > fb * (1.0f + 1e-4f)) return 0;
    }
    return -1;
}

__global__ void k_cand(int level, int step, int64_t npar, double theta, const int32_t *__restrict__ pptr,
                       const int32_t *__restrict__ psrc, const int32_t *__restrict__ prow,
                       const double *__restrict__ centre, const double *__restrict__ radius,
                       const float4 *__restrict__ cf, int32_t *__restrict__ flag, int32_t *__restrict__ csrc,
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
            int w = theta > 0.0 ? theta_pretest((float)theta, cf[2 * gt], cf[2 * gt + 1], cf[2 * gs], cf[2 * gs + 1])
                                : 0;
            if (w < 0) w = theta_weak(theta, centre + 3 * gt, radius[gt], centre + 3 * gs, radius[gs]) ? 1 : 0;
            flag[base + b] = w;
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
// pairs), and in total the sum over strong leaf pairs (t, s) of n_t * n_s.
// Per leaf: its sources over the strong list, its number of near-field work
// units -- tiles of `tile` targets times k source segments, k = ceil(sources /
// smax) -- and, when k > 1, the k * n_t partial-sum slots its split units fill;
// the totals (pairs, units, slots) into acc[0..2] in 64 bits. One warp per
// leaf, its lanes striding over the strong list (lists of large boxes in
// sparse regions hold a good part of the tree).
__global__ void k_p2p_work(int B, int tile, long long smax, const int32_t *sptr, const int32_t *ssrc,
                           const int32_t *count, unsigned long long *acc, long long *per_leaf,
                           int32_t *units_per_leaf, int32_t *parts_per_leaf) {
    const int64_t nt = (int64_t)1 << B, off = nt - 1;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long v = 0, vu = 0, vp = 0;  // this warp's totals (lane 0)
    for (int64_t t = warp; t < nt; t += nwarps) {
        unsigned long long ns = 0;
        const int e1 = sptr[t + 1];
#pragma unroll 4
        for (int e = sptr[t] + lane; e < e1; e += 32) ns += (unsigned long long)count[off + ssrc[e]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ns += __shfl_xor_sync(0xffffffffu, ns, o);
        if (lane == 0) {
            const int n_t = count[off + t];
            per_leaf[t] = (long long)ns;
            const unsigned long long k = ns > (unsigned long long)smax ? (ns + smax - 1) / smax : 1;
            const unsigned long long u = (unsigned long long)((n_t + tile - 1) / tile) * k;
            const unsigned long long pp = k > 1 ? k * (unsigned long long)n_t : 0;
            // stored as int32; the host rejects the plan if a total exceeds 2^31 - 1
            units_per_leaf[t] = (int32_t)min(u, 0x7fffffffull);
            parts_per_leaf[t] = (int32_t)min(pp, 0x7fffffffull);
            v += ns * (unsigned long long)n_t;
            vu += u;
            vp += pp;
        }
    }
    if (lane == 0) {
        if (v) atomicAdd(acc, v);
        if (vu) atomicAdd(acc + 1, vu);
        if (vp) atomicAdd(acc + 2, vp);
    }
}

// Work units heaviest first, on the device: each unit's weight (targets x the
// leaf's sources) is quantised to a quarter-octave bucket (0 = heaviest), and a
// stable counting sort over the buckets orders them (within a bucket, leaf
// order). The exact order only affects the near field's load balance.
constexpr int kUnitBlock = 256;
__device__ __forceinline__ int unit_bucket(unsigned long long w) {
    if (w == 0) return 255;
    const int lg = 63 - __clzll((long long)w);
    const int frac = lg >= 2 ? (int)((w >> (lg - 2)) & 3ull) : (int)((w << (2 - lg)) & 3ull);
    return 255 - min(255, 4 * lg + frac);
}

constexpr int kUnitPre = 8;

// One warp per leaf: cuts the leaf's strong list into k segments of about
// nsrc / k sources each and emits its units (leaf, first target, segment
// begin, segment end) with their partial-sum slot (-1 when the leaf is not
// split) and weight bucket. Segment j ends just after the first list entry
// at which the cumulative source count reaches floor((j + 1) nsrc / k) (the
// last one at the list's end); the lanes scan 32 entries at a time and a
// ballot finds the entry for each such goal.
__global__ void k_units_gen(int B, int tile, long long smax, const int32_t *count, const long long *nsrc,
                            const int32_t *sptr, const int32_t *ssrc, const int32_t *uoff,
                            const int32_t *poff, int4 *units, int32_t *upart, uint8_t *bucket) {
    const int64_t nt = (int64_t)1 << B, off = nt - 1;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < nt; t += nwarps) {
        const int cnt = count[off + t];
        if (cnt == 0) continue;
        const long long ns = nsrc[t];
        const int k = ns > smax ? (int)((ns + smax - 1) / smax) : 1;
        const int ntile = (cnt + tile - 1) / tile;
        const int l0 = sptr[t], l1 = sptr[t + 1];
        // emits segment j = [e_lo, e_hi) holding w sources (lanes over its tiles)
        auto emit = [&](int j, int e_lo, int e_hi, long long w) {
            for (int ti = lane; ti < ntile; ti += 32) {
                const int u = uoff[t] + j * ntile + ti, tb = ti * tile;
                units[u] = make_int4((int)t, tb, e_lo, e_hi);
                upart[u] = k > 1 ? poff[t] + j * cnt : -1;
                bucket[u] = (uint8_t)unit_bucket((unsigned long long)min(tile, cnt - tb) * (unsigned long long)w);
            }
        };
        if (k == 1) {
            emit(0, l0, l1, ns);
            continue;
        }
        int j = 0, e_lo = l0;
        long long c_lo = 0, run = 0;  // cumulative sources before the chunk
        // chunks of 32 entries; the source counts of kUnitPre chunks are
        // fetched together (two dependent loads each), so that a long list
        // waits on memory once per kUnitPre chunks
        for (int base0 = l0; base0 < l1 && j < k - 1; base0 += 32 * kUnitPre) {
            long long cn[kUnitPre];
#pragma unroll
            for (int u = 0; u < kUnitPre; u++) {
                const int e = base0 + 32 * u + lane;
                cn[u] = e < l1 ? (long long)count[off + ssrc[e]] : 0;
            }
#pragma unroll
            for (int u = 0; u < kUnitPre; u++) {
                const int base = base0 + 32 * u;
                if (base >= l1 || j >= k - 1) break;  // warp-uniform
                const int e = base + lane;
                long long c = cn[u];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {  // inclusive scan over the chunk
                    const long long y = __shfl_up_sync(0xffffffffu, c, o);
                    if (lane >= o) c += y;
                }
                const long long total = __shfl_sync(0xffffffffu, c, 31);
                while (j < k - 1) {
                    const long long goal = (long long)(((unsigned long long)ns * (unsigned long long)(j + 1)) / k);
                    const unsigned hit = __ballot_sync(0xffffffffu, e < l1 && run + c >= goal);
                    if (!hit) break;
                    const int f = __ffs(hit) - 1;
                    const int e_hi = base + f + 1;
                    const long long c_hi = run + __shfl_sync(0xffffffffu, c, f);
                    emit(j, e_lo, e_hi, c_hi - c_lo);
                    e_lo = e_hi;
                    c_lo = c_hi;
                    j++;
                }
                run += total;
            }
        }
        for (; j < k; j++) {  // the last segment (and any left empty) end at the list's end
            emit(j, e_lo, l1, ns - c_lo);
            e_lo = l1;
            c_lo = ns;
        }
    }
}

// counts per (bucket, block of kUnitBlock units), bucket-major
__global__ void __launch_bounds__(kUnitBlock)
k_units_hist(const int32_t *total, const uint8_t *bucket, int nblocks, int32_t *bh) {
    __shared__ int32_t h[256];
    const int tid = threadIdx.x, k = blockIdx.x;
    h[tid] = 0;
    __syncthreads();
    const int u = k * kUnitBlock + tid;
    if (u < *total) atomicAdd(&h[bucket[u]], 1);
    __syncthreads();
    bh[(int64_t)tid * nblocks + k] = h[tid];
}

// stable scatter: a unit's place is its bucket's offset for its block plus the
// units of the same bucket before it in the block (warp match, then warps)
__global__ void __launch_bounds__(kUnitBlock)
k_units_scatter(const int32_t *total, const uint8_t *bucket, const int4 *units, const int32_t *upart,
                int nblocks, const int32_t *boff, int4 *sorted, int32_t *sorted_part) {
    __shared__ int32_t wc[kUnitBlock / 32][256];
    const int tid = threadIdx.x, k = blockIdx.x, lane = tid & 31, w = tid >> 5;
    for (int i = tid; i < (kUnitBlock / 32) * 256; i += kUnitBlock) (&wc[0][0])[i] = 0;
    __syncthreads();
    const int u = k * kUnitBlock + tid;
    const bool valid = u < *total;
    const int b = valid ? bucket[u] : 256;  // 256: no bucket
    const unsigned same = __match_any_sync(0xffffffffu, b);
    const int rank_w = __popc(same & ((1u << lane) - 1u));
    if (valid && rank_w == 0) wc[w][b] = __popc(same);
    __syncthreads();
    if (valid) {
        int r = boff[(int64_t)b * nblocks + k] + rank_w;
        for (int j = 0; j < w; j++) r += wc[j][b];
        sorted[r] = units[u];
        sorted_part[r] = upart[u];
    }
}

// first sorted unit of each weight bucket (bstart[256] = the unit count)
__global__ void k_bucket_starts(const int32_t *boff, int nblocks, const int32_t *total, int32_t *bstart) {
    const int b = threadIdx.x;
    bstart[b] = boff[(int64_t)b * nblocks];
    if (b == 0) bstart[256] = *total;
}

}  // namespace

namespace {
// the theta-criterion of the list build, on n given box pairs
__global__ void k_theta_pairs(double theta, int64_t n, const double *ca, const double *ra, const double *cb,
                              const double *rb, uint8_t *weak) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        weak[i] = theta_weak(theta, ca + 3 * i, ra[i], cb + 3 * i, rb[i]) ? 1 : 0;
}
}  // namespace

cudaError_t theta_pairs(double theta, int64_t n, const double *ca, const double *ra, const double *cb,
                        const double *rb, uint8_t *weak, cudaStream_t st) {
    if (n == 0) return cudaGetLastError();
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
    FMM_LAUNCH(k_theta_pairs, grid, 256, 0, st, theta, n, ca, ra, cb, rb, weak);
    return cudaGetLastError();
}

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

// Largest candidate-pair array a level may need (entries): the lists index
// it with int32. Lowered only by fmm_set_list_capacity (tests).
std::atomic<long long> g_list_capacity{0x7fffffffLL};

cudaError_t lists_build(Plan &P) {
    cudaStream_t st = P.stream;
    // every box's centre split hi + lo in float and its radius, for the
    // theta-test's single-precision pre-test (and the single-precision M2L)
    P.box_cf = (float4 *)palloc(P, (size_t)P.nbox * 2 * sizeof(float4));
    if (!P.box_cf) return cudaErrorMemoryAllocation;
    box_centres_f(P);
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
        if (ncand > g_list_capacity.load(std::memory_order_relaxed)) {
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
                   P.ssrc[lp], srow_prev, P.centre, P.radius, P.box_cf, flag, csrc, ctgt);
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
    // field runs as work units of up to `tile` targets of one leaf against a
    // segment of its strong list of at most about kP2PSegSources sources, so
    // that neither a few large leaves nor the leaves strongly connected to
    // most of the tree (large boxes in sparse regions of clustered inputs)
    // leave the GPU waiting on a handful of blocks; units go heaviest first,
    // so that the long ones start early instead of forming the tail of the
    // launch. A leaf cut into k segments gets k partial sums per target,
    // added in segment order by the combine pass. The unit and slot totals
    // are read back once to size the arrays.
    const int64_t nl = (int64_t)1 << P.B;
    P.p2p_tile = (P.prec == FMM_PREC_MIXED && P.n <= (int64_t)kP2PTileSmall * nl) ? kP2PTileSmall : kP2PTile;
    const int tile = P.p2p_tile;
    P.p2p_work_dev = (unsigned long long *)palloc(P, 24);  // pairs, units, partial slots
    long long *nsrc = (long long *)dalloc(P, (size_t)nl * 8);
    int32_t *upl = (int32_t *)dalloc(P, (size_t)nl * 4);
    int32_t *ppl = (int32_t *)dalloc(P, (size_t)nl * 4);
    int32_t *uoff = (int32_t *)palloc(P, (size_t)(nl + 1) * 4);  // its total is read at evaluation
    P.p2p_poff = (int32_t *)palloc(P, (size_t)(nl + 1) * 4);
    if (!P.p2p_work_dev || !nsrc || !upl || !ppl || !uoff || !P.p2p_poff) return cudaErrorMemoryAllocation;
    cudaMemsetAsync(P.p2p_work_dev, 0, 24, st);
    const unsigned wgrid = (unsigned)std::min<int64_t>((nl * 32 + 255) / 256, (int64_t)sm_count() * 32);
    FMM_LAUNCH(k_p2p_work, wgrid, 256, 0, st, P.B, tile, (long long)kP2PSegSources,
               P.sptr[P.B], P.ssrc[P.B], P.count, P.p2p_work_dev, nsrc, upl, ppl);
    e = scan_exclusive(P, upl, uoff, nl);
    if (e == cudaSuccess) e = scan_exclusive(P, ppl, P.p2p_poff, nl);
    if (e != cudaSuccess) return e;
    unsigned long long tot[3] = {0, 0, 0};
    cudaMemcpyAsync(tot, P.p2p_work_dev, 24, cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (tot[1] > 0x7fffffffull || tot[2] > 0x7fffffffull) {  // the int32 scans would overflow
        P.capacity_exceeded = true;
        return cudaSuccess;
    }
    const int64_t nunits = (int64_t)tot[1];
    P.p2p_nparts = (int64_t)tot[2];
    const int nblk = (int)std::max<int64_t>((nunits + kUnitBlock - 1) / kUnitBlock, 1);
    int4 *units = (int4 *)dalloc(P, (size_t)std::max<int64_t>(nunits, 1) * sizeof(int4));
    int32_t *upart = (int32_t *)dalloc(P, (size_t)std::max<int64_t>(nunits, 1) * 4);
    uint8_t *bucket = (uint8_t *)dalloc(P, (size_t)std::max<int64_t>(nunits, 1));
    int32_t *bh = (int32_t *)dalloc(P, (size_t)256 * nblk * 4);
    int32_t *boff = (int32_t *)dalloc(P, ((size_t)256 * nblk + 1) * 4);
    P.p2p_units = (int4 *)palloc(P, (size_t)std::max<int64_t>(nunits, 1) * sizeof(int4));
    P.p2p_upart = (int32_t *)palloc(P, (size_t)std::max<int64_t>(nunits, 1) * 4);
    P.p2p_partial = P.p2p_nparts ? (double4 *)palloc(P, (size_t)P.p2p_nparts * sizeof(double4)) : nullptr;
    P.p2p_bstart = (int32_t *)palloc(P, 257 * 4);
    if (!units || !upart || !bucket || !bh || !boff || !P.p2p_units || !P.p2p_upart || !P.p2p_bstart ||
        (P.p2p_nparts && !P.p2p_partial))
        return cudaErrorMemoryAllocation;
    P.p2p_nunits_dev = uoff + nl;
    P.p2p_nunits = nunits;
    FMM_LAUNCH(k_units_gen, wgrid, 256, 0, st, P.B, tile, (long long)kP2PSegSources,
               P.count, nsrc, P.sptr[P.B], P.ssrc[P.B], uoff, P.p2p_poff, units, upart, bucket);
    FMM_LAUNCH(k_units_hist, (unsigned)nblk, kUnitBlock, 0, st, P.p2p_nunits_dev, bucket, nblk, bh);
    e = scan_exclusive(P, bh, boff, (int64_t)256 * nblk);
    if (e != cudaSuccess) return e;
    FMM_LAUNCH(k_units_scatter, (unsigned)nblk, kUnitBlock, 0, st, P.p2p_nunits_dev, bucket, units, upart, nblk,
               boff, P.p2p_units, P.p2p_upart);
    FMM_LAUNCH(k_bucket_starts, 1, 256, 0, st, boff, nblk, P.p2p_nunits_dev, P.p2p_bstart);
    return cudaGetLastError();
}

}  // namespace fmm

extern "C" int64_t fmm_set_list_capacity(int64_t entries) {
    if (entries < 1 || entries > 0x7fffffffLL) entries = 0x7fffffffLL;
    return (int64_t)fmm::g_list_capacity.exchange(entries);
}
