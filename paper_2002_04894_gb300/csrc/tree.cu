// Balanced-tree construction (Sec. 2.1.2 with eta = 1; Algorithm 2 on one
// device): the root cell is the tight bounding box of the points; every box of
// a level is split on the longest axis of its cell so that the left child
// receives the floor(n/2) smallest (coordinate, original index) keys, both
// children keeping ascending original-index order; the split plane lies
// halfway between the largest left and the smallest right coordinate.
//
// GPU design. Points are kept in structure-of-arrays order (x | y | z | idx)
// and ping-pong between two buffers, one level per pass. Because the tree is
// balanced, every segment of a level holds floor or ceil(N / 2^l) points, so a
// level is handled by one of two regimes:
//   small  (<= 4096 points per box): one CTA per box, keys in shared memory,
//          8-bit radix select of the rank-(k-1) key, then a warp-ballot stable
//          partition;
//   large: many CTAs per box (4096-point chunks); per-pass histograms are
//          privatised in shared memory and merged with global atomics, a
//          one-warp pick kernel chooses each digit, and the stable partition
//          is a chunk-level count, a per-box scan of chunk counts and a
//          warp-ballot scatter.
// Keys are order-preserving 64-bit images of the coordinate. Since a box's
// points are in ascending original index, the index tie-break of the key
// (coordinate, index) equals the position order inside the box: among points
// equal to the selected key v, the first (k - #{key < v}) in position go left.
// All geometry uses explicitly rounded double operations (no contraction).

#include <algorithm>
#include <utility>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kSmallCap = 4096;
constexpr int kChunk = 4096;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t t = __shfl_xor_sync(0xffffffffu, v, o);
        v = t < v ? t : v;
    }
    return v;
}

// Cell geometry of box g: centre = 0.5 (lo + hi); radius = 0.5 sqrt((ex^2 + ey^2) + ez^2);
// split axis = first longest extent.
__device__ void box_geometry(double *lo, double *hi, double *centre, double *radius,
                             int32_t *axis, int64_t g) {
    double e[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        e[a] = __dsub_rn(hi[3 * g + a], lo[3 * g + a]);
        centre[3 * g + a] = __dmul_rn(0.5, __dadd_rn(lo[3 * g + a], hi[3 * g + a]));
    }
    double s = __dadd_rn(__dadd_rn(__dmul_rn(e[0], e[0]), __dmul_rn(e[1], e[1])),
                         __dmul_rn(e[2], e[2]));
    radius[g] = __dmul_rn(0.5, __dsqrt_rn(s));
    int ax = 0;
    if (e[1] > e[ax]) ax = 1;
    if (e[2] > e[ax]) ax = 2;
    axis[g] = ax;
}

// --------------------------------------------------------------------------
// Input: n x 3 row-major -> SoA doubles, -0.0 -> +0.0, finiteness, bounding box
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_prepare(const T *__restrict__ pts, int64_t n, double *__restrict__ x, double *__restrict__ y,
          double *__restrict__ z, int32_t *__restrict__ idx, unsigned long long *bbox, int *err) {
    uint64_t mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            v[a] = (double)pts[3 * i + a] + 0.0;
            bad |= !isfinite(v[a]);
            uint64_t k = dkey(v[a]);
            mn[a] = k < mn[a] ? k : mn[a];
            mx[a] = k > mx[a] ? k : mx[a];
        }
        x[i] = v[0];
        y[i] = v[1];
        z[i] = v[2];
        idx[i] = (int32_t)i;
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        mn[a] = warp_min_u64(mn[a]);
        for (int o = 16; o > 0; o >>= 1) {
            uint64_t t = __shfl_xor_sync(0xffffffffu, mx[a], o);
            mx[a] = t > mx[a] ? t : mx[a];
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, 1);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            atomicMin(&bbox[a], (unsigned long long)mn[a]);
            atomicMax(&bbox[3 + a], (unsigned long long)mx[a]);
        }
    }
}

// The root cell: the points' bounding box, or a given cell (FMM_FLAG_ROOT_CELL:
// a box of a larger tree, so that this tree is that box's subtree) that must
// hold every point (else error bit 4).
__global__ void k_root(const unsigned long long *bbox, RootCell rc, double *lo, double *hi, double *centre,
                       double *radius, int32_t *axis, int *err) {
    if (threadIdx.x != 0) return;
    for (int a = 0; a < 3; a++) {
        if (rc.given) {
            lo[a] = rc.lo[a] + 0.0;  // -0.0 -> +0.0, as the points
            hi[a] = rc.hi[a] + 0.0;
            if (dkey(lo[a]) > bbox[a] || bbox[3 + a] > dkey(hi[a])) atomicOr(err, 4);
        } else {
            lo[a] = dkey_inv(bbox[a]);
            hi[a] = dkey_inv(bbox[3 + a]);
        }
    }
    box_geometry(lo, hi, centre, radius, axis, 0);
}

// --------------------------------------------------------------------------
// Shared pieces of the radix select
// --------------------------------------------------------------------------

// One warp: find the digit whose bucket holds rank *rrem among hist[0..255],
// update the key prefix and the remaining rank.
// (cnt, when given, receives the number of keys in the chosen bucket)
__device__ void pick_digit(const unsigned *hist, int shift, uint64_t *prefix, unsigned *rrem,
                           unsigned *cnt = nullptr) {
    const int lane = threadIdx.x & 31;
    unsigned c[8], sum = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        c[j] = hist[lane * 8 + j];
        sum += c[j];
    }
    unsigned incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const unsigned excl = incl - sum;
    const unsigned r = *rrem;
    const uint64_t pre = *prefix;
    __syncwarp();
    if (excl <= r && r < incl) {
        unsigned acc = excl;
        for (int j = 0; j < 8; j++) {
            if (r < acc + c[j]) {
                *rrem = r - acc;
                *prefix = pre | ((uint64_t)(lane * 8 + j) << shift);
                if (cnt) *cnt = c[j];
                break;
            }
            acc += c[j];
        }
    }
    __syncwarp();
}

__device__ __forceinline__ bool prefix_match(uint64_t key, uint64_t prefix, int shift) {
    return shift >= 56 || (key >> (shift + 8)) == (prefix >> (shift + 8));
}

// --------------------------------------------------------------------------
// Small regime: one CTA per box
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_split_small(int level, const double *__restrict__ xin, const double *__restrict__ yin,
              const double *__restrict__ zin, const int32_t *__restrict__ iin,
              double *__restrict__ xout, double *__restrict__ yout, double *__restrict__ zout,
              int32_t *__restrict__ iout, const int32_t *__restrict__ begin,
              const int32_t *__restrict__ count, const int32_t *__restrict__ axis,
              uint64_t *sel_v, unsigned long long *sel_minr, int *err,
              const unsigned long long *__restrict__ thr, int32_t *__restrict__ ksplit) {
    // thr == nullptr: median split (left = floor(n/2) smallest keys);
    // otherwise threshold split (left = keys below thr[s], count to ksplit[s])
    __shared__ uint64_t keys[kSmallCap];
    __shared__ unsigned hist[256];
    __shared__ unsigned flags[kSmallCap / 32];
    __shared__ uint64_t s_prefix;
    __shared__ unsigned s_rrem;
    __shared__ unsigned long long s_minr;
    __shared__ unsigned w_eq[kWarps], w_left[kWarps];
    __shared__ bool s_one;

    const int s = blockIdx.x;
    const int64_t g = ((int64_t)1 << level) - 1 + s;
    const int b = begin[g], n = count[g], ax = axis[g];
    int k = n / 2;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const double *src = ax == 0 ? xin : (ax == 1 ? yin : zin);

    if (n <= 1) {
        if (n == 1 && tid == 0) {
            xout[b] = xin[b];
            yout[b] = yin[b];
            zout[b] = zin[b];
            iout[b] = iin[b];
            if (thr) {
                ksplit[s] = dkey(src[b]) < thr[s] ? 1 : 0;
            } else {
                sel_v[s] = dkey(src[b]);
                sel_minr[s] = dkey(src[b]);
            }
        }
        if (n == 0 && thr && tid == 0) ksplit[s] = 0;
        return;
    }
    for (int i = tid; i < n; i += kThreads) keys[i] = dkey(src[b + i]);
    if (tid == 0) {
        s_prefix = 0;
        s_rrem = (unsigned)(k - 1);
        s_minr = ~0ull;
    }
    __syncthreads();

    for (int pass = 0; pass < 8 && !thr; pass++) {
        const int shift = 56 - 8 * pass;
        hist[tid] = 0;  // kThreads == 256 bins
        __syncthreads();
        const uint64_t pre = s_prefix;
        for (int i = tid; i < n; i += kThreads) {
            uint64_t kk = keys[i];
            if (prefix_match(kk, pre, shift)) atomicAdd(&hist[(kk >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (w == 0) {
            unsigned c = 0;
            pick_digit(hist, shift, &s_prefix, &s_rrem, &c);
            c = __reduce_max_sync(0xffffffffu, c);  // the picking lane's bucket count
            if (lane == 0) s_one = c == 1u;
        }
        __syncthreads();
        if (s_one && pass < 7) {  // one key under the prefix: it is the wanted one
            const uint64_t pre2 = s_prefix;
            for (int i = tid; i < n; i += kThreads) {
                const uint64_t kk = keys[i];
                if ((kk >> shift) == (pre2 >> shift)) s_prefix = kk;
            }
            __syncthreads();
            break;
        }
    }
    const uint64_t v = thr ? (uint64_t)thr[s] : s_prefix;
    const unsigned need_eq = thr ? 0u : s_rrem + 1;  // equal keys that go left, in position order

    // warp w owns positions [start, end)
    const int per_warp = ((n + kWarps - 1) / kWarps + 31) & ~31;
    const int start = w * per_warp;
    const int end = min(n, start + per_warp);

    unsigned eqc = 0;
    uint64_t mr = ~0ull;
    for (int base = start; base < end; base += 32) {
        const int i = base + lane;
        const bool valid = i < end;
        const uint64_t kk = valid ? keys[i] : 0;
        eqc += __popc(__ballot_sync(0xffffffffu, valid && kk == v));
        if (valid && kk > v && kk < mr) mr = kk;
    }
    mr = warp_min_u64(mr);
    if (lane == 0) {
        w_eq[w] = eqc;
        atomicMin(&s_minr, (unsigned long long)mr);
    }
    __syncthreads();
    unsigned eqrun = 0, eqtot = 0;
    for (int j = 0; j < kWarps; j++) {
        eqrun += j < w ? w_eq[j] : 0;
        eqtot += w_eq[j];
    }
    unsigned leftc = 0;
    for (int base = start; base < end; base += 32) {
        const int i = base + lane;
        const bool valid = i < end;
        const uint64_t kk = valid ? keys[i] : 0;
        const bool eq = valid && kk == v;
        const unsigned em = __ballot_sync(0xffffffffu, eq);
        const unsigned rank = eqrun + __popc(em & lanemask_lt());
        const bool f = valid && (kk < v || (eq && rank < need_eq));
        const unsigned fm = __ballot_sync(0xffffffffu, f);
        if (lane == 0) flags[base >> 5] = fm;
        leftc += __popc(fm);
        eqrun += __popc(em);
    }
    if (lane == 0) w_left[w] = leftc;
    __syncthreads();
    unsigned lrun = 0;
    for (int j = 0; j < w; j++) lrun += w_left[j];
    if (thr) {
        k = 0;
        for (int j = 0; j < kWarps; j++) k += w_left[j];
        if (tid == 0) ksplit[s] = k;
    }
    for (int base = start; base < end; base += 32) {
        const int i = base + lane;
        const unsigned fm = flags[base >> 5];
        const bool f = (fm >> lane) & 1u;
        const unsigned lrank = lrun + __popc(fm & lanemask_lt());
        if (i < end) {
            const int rel = f ? (int)lrank : k + (i - (int)lrank);
            if (rel >= 0 && rel < n) {
                xout[b + rel] = xin[b + i];
                yout[b + rel] = yin[b + i];
                zout[b + rel] = zin[b + i];
                iout[b + rel] = iin[b + i];
            } else {
                atomicOr(err, 2);  // inconsistent partition: report, never write outside the box
            }
        }
        lrun += __popc(fm);
    }
    if (tid == 0 && !thr) {
        sel_v[s] = v;
        sel_minr[s] = eqtot > need_eq ? (unsigned long long)v : s_minr;
    }
}

// --------------------------------------------------------------------------
// Large regime: many CTAs per box
// --------------------------------------------------------------------------
__global__ void k_sel_init(int level, const int32_t *count, uint64_t *prefix, unsigned *rrem,
                           unsigned long long *minr, unsigned *ghist, unsigned *found) {
    const int s = blockIdx.x;
    const int64_t g = ((int64_t)1 << level) - 1 + s;
    if (threadIdx.x == 0) {
        const int n = count[g];
        prefix[s] = 0;
        rrem[s] = n >= 2 ? (unsigned)(n / 2 - 1) : 0u;
        minr[s] = ~0ull;
        found[s] = 0;
    }
    for (int i = threadIdx.x; i < 256; i += blockDim.x) ghist[(int64_t)s * 256 + i] = 0;
}

// One chunk of one box: histogram of the keys' current digit, added to the
// box's global histogram. The last chunk of the box to finish (a per-box
// arrival counter) then picks the digit holding the wanted rank, clears the
// histogram and the counter for the next pass. When the chosen bucket holds
// a single key (found = 1), the next pass just finds that key (found = 2) and
// the remaining passes of the box return at once.
__global__ void __launch_bounds__(kThreads)
k_sel_hist(int level, int pass, const double *__restrict__ xs, const double *__restrict__ ys,
           const double *__restrict__ zs, const int32_t *__restrict__ begin,
           const int32_t *__restrict__ count, const int32_t *__restrict__ axis,
           uint64_t *prefix, unsigned *rrem, unsigned *ghist, unsigned *arrived, unsigned *found) {
    __shared__ unsigned h[256];
    __shared__ bool last;
    __shared__ uint64_t s_pre;
    __shared__ unsigned s_rr;
    const int s = blockIdx.x, c = blockIdx.y;
    const int64_t g = ((int64_t)1 << level) - 1 + s;
    const int b = begin[g], n = count[g], ax = axis[g];
    const int start = c * kChunk;
    if (start >= n) return;
    const int end = min(n, start + kChunk);
    const double *src = ax == 0 ? xs : (ax == 1 ? ys : zs);
    const unsigned state = found[s];  // uniform over the block
    if (state == 2u) return;
    const int shift = 56 - 8 * pass;
    const uint64_t pre = prefix[s];
    if (state == 1u) {  // the one key under the prefix is the wanted one
        for (int i = start + threadIdx.x; i < end; i += kThreads) {
            const uint64_t kk = dkey(src[b + i]);
            if (prefix_match(kk, pre, shift)) {
                prefix[s] = kk;
                found[s] = 2u;
            }
        }
        return;
    }
    h[threadIdx.x] = 0;
    __syncthreads();
    for (int i = start + threadIdx.x; i < end; i += kThreads) {
        const uint64_t kk = dkey(src[b + i]);
        if (prefix_match(kk, pre, shift)) atomicAdd(&h[(kk >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&ghist[(int64_t)s * 256 + threadIdx.x], h[threadIdx.x]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned active = (unsigned)((n + kChunk - 1) / kChunk);
        last = atomicAdd(&arrived[s], 1u) == active - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    h[threadIdx.x] = __ldcg(&ghist[(int64_t)s * 256 + threadIdx.x]);
    ghist[(int64_t)s * 256 + threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        s_pre = prefix[s];
        s_rr = rrem[s];
        arrived[s] = 0;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned c = 0;
        pick_digit(h, shift, &s_pre, &s_rr, &c);
        if (threadIdx.x == 0) {
            prefix[s] = s_pre;
            rrem[s] = s_rr;
        }
        // the lane that picked wrote c; bring it to lane 0
        c = __reduce_max_sync(0xffffffffu, c);
        if (threadIdx.x == 0 && c == 1u && pass < 7) found[s] = 1u;
    }
}

__global__ void __launch_bounds__(kThreads)
k_sel_count(int level, int nch, const double *__restrict__ xs, const double *__restrict__ ys,
            const double *__restrict__ zs, const int32_t *__restrict__ begin,
            const int32_t *__restrict__ count, const int32_t *__restrict__ axis,
            const uint64_t *__restrict__ prefix, unsigned *chunk_lt, unsigned *chunk_eq,
            unsigned long long *minr, const unsigned long long *__restrict__ thr) {
    __shared__ unsigned s_lt[kWarps], s_eq[kWarps];
    __shared__ unsigned long long s_mr;
    const int s = blockIdx.x, c = blockIdx.y;
    const int64_t g = ((int64_t)1 << level) - 1 + s;
    const int b = begin[g], n = count[g], ax = axis[g];
    const int start = c * kChunk;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_mr = ~0ull;
    __syncthreads();
    const double *src = ax == 0 ? xs : (ax == 1 ? ys : zs);
    const uint64_t v = thr ? (uint64_t)thr[s] : prefix[s];
    unsigned lt = 0, eq = 0;
    uint64_t mr = ~0ull;
    const int end = min(n, start + kChunk);
    for (int i = start + threadIdx.x; i < end; i += kThreads) {
        const uint64_t kk = dkey(src[b + i]);
        lt += kk < v;
        eq += kk == v;
        if (kk > v && kk < mr) mr = kk;
    }
    for (int o = 16; o > 0; o >>= 1) {
        lt += __shfl_xor_sync(0xffffffffu, lt, o);
        eq += __shfl_xor_sync(0xffffffffu, eq, o);
    }
    mr = warp_min_u64(mr);
    if (lane == 0) {
        s_lt[w] = lt;
        s_eq[w] = eq;
        atomicMin(&s_mr, (unsigned long long)mr);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned a = 0, e = 0;
        for (int j = 0; j < kWarps; j++) a += s_lt[j], e += s_eq[j];
        chunk_lt[(int64_t)s * nch + c] = a;
        chunk_eq[(int64_t)s * nch + c] = e;
        if (s_mr != ~0ull) atomicMin(&minr[s], s_mr);
    }
}

// Per box: exclusive scans over its chunks of the equal-key counts and of the
// left counts; fixes the smallest right key when equal keys straddle.
__global__ void k_sel_offsets(int level, int nch, const int32_t *count, const unsigned *chunk_lt,
                              const unsigned *chunk_eq, const uint64_t *prefix,
                              const unsigned *rrem, unsigned *eq_off, unsigned *left_off,
                              unsigned long long *minr, uint64_t *sel_v,
                              const unsigned long long *thr, int32_t *ksplit) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= (1 << level)) return;
    const unsigned need_eq = thr ? 0u : rrem[s] + 1;
    unsigned eo = 0, lo = 0;
    for (int c = 0; c < nch; c++) {
        const int64_t i = (int64_t)s * nch + c;
        const unsigned e = chunk_eq[i], l = chunk_lt[i];
        eq_off[i] = eo;
        left_off[i] = lo;
        const unsigned take = need_eq > eo ? min(need_eq - eo, e) : 0u;
        lo += l + take;
        eo += e;
    }
    if (thr) {
        ksplit[s] = (int32_t)lo;
        return;
    }
    sel_v[s] = prefix[s];
    if (eo > need_eq) minr[s] = prefix[s];
}

__global__ void __launch_bounds__(kThreads)
k_sel_scatter(int level, int nch, const double *__restrict__ xin, const double *__restrict__ yin,
              const double *__restrict__ zin, const int32_t *__restrict__ iin,
              double *__restrict__ xout, double *__restrict__ yout, double *__restrict__ zout,
              int32_t *__restrict__ iout, const int32_t *__restrict__ begin,
              const int32_t *__restrict__ count, const int32_t *__restrict__ axis,
              const uint64_t *__restrict__ prefix, const unsigned *__restrict__ rrem,
              const unsigned *__restrict__ eq_off, const unsigned *__restrict__ left_off, int *err,
              const unsigned long long *__restrict__ thr, const int32_t *__restrict__ ksplit) {
    __shared__ unsigned flags[kChunk / 32];
    __shared__ unsigned w_eq[kWarps], w_left[kWarps];
    const int s = blockIdx.x, c = blockIdx.y;
    const int64_t g = ((int64_t)1 << level) - 1 + s;
    const int b = begin[g], n = count[g], ax = axis[g];
    const int k = thr ? ksplit[s] : n / 2;
    const int cstart = c * kChunk;
    if (cstart >= n) return;
    const int cend = min(n, cstart + kChunk);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const double *src = ax == 0 ? xin : (ax == 1 ? yin : zin);
    const uint64_t v = thr ? (uint64_t)thr[s] : prefix[s];
    const unsigned need_eq = thr ? 0u : rrem[s] + 1;
    constexpr int per_warp = kChunk / kWarps;
    const int start = cstart + w * per_warp;
    const int end = min(cend, start + per_warp);

    unsigned eqc = 0;
    for (int base = start; base < end; base += 32) {
        const int i = base + lane;
        const bool valid = i < end;
        const uint64_t kk = valid ? dkey(src[b + i]) : 0;
        eqc += __popc(__ballot_sync(0xffffffffu, valid && kk == v));
    }
    if (lane == 0) w_eq[w] = eqc;
    __syncthreads();
    unsigned eqrun = eq_off[(int64_t)s * nch + c];
    for (int j = 0; j < w; j++) eqrun += w_eq[j];
    unsigned leftc = 0;
    for (int base = start; base < end; base += 32) {
        const int i = base + lane;
        const bool valid = i < end;
        const uint64_t kk = valid ? dkey(src[b + i]) : 0;
        const bool eq = valid && kk == v;
        const unsigned em = __ballot_sync(0xffffffffu, eq);
        const unsigned rank = eqrun + __popc(em & lanemask_lt());
        const bool f = valid && (kk < v || (eq && rank < need_eq));
        const unsigned fm = __ballot_sync(0xffffffffu, f);
        if (lane == 0) flags[(base - cstart) >> 5] = fm;
        leftc += __popc(fm);
        eqrun += __popc(em);
    }
    if (lane == 0) w_left[w] = leftc;
    __syncthreads();
    unsigned lrun = left_off[(int64_t)s * nch + c];
    for (int j = 0; j < w; j++) lrun += w_left[j];
    for (int base = start; base < end; base += 32) {
        const int i = base + lane;
        const unsigned fm = flags[(base - cstart) >> 5];
        const bool f = (fm >> lane) & 1u;
        const unsigned lrank = lrun + __popc(fm & lanemask_lt());
        if (i < end) {
            const int rel = f ? (int)lrank : k + (i - (int)lrank);
            if (rel >= 0 && rel < n) {
                xout[b + rel] = xin[b + i];
                yout[b + rel] = yin[b + i];
                zout[b + rel] = zin[b + i];
                iout[b + rel] = iin[b + i];
            } else {
                atomicOr(err, 2);  // inconsistent partition: report, never write outside the box
            }
        }
        lrun += __popc(fm);
    }
}

// --------------------------------------------------------------------------
// Children's cells and geometry
// --------------------------------------------------------------------------
__global__ void k_children(int level, const int32_t *count, const uint64_t *sel_v,
                           const unsigned long long *sel_minr, double *lo, double *hi, double *centre,
                           double *radius, int32_t *axis, double *plane) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= (1 << level)) return;
    const int64_t g = ((int64_t)1 << level) - 1 + s;
    const int n = count[g], ax = axis[g];
    double sp;
    if (n >= 2)
        sp = __dmul_rn(0.5, __dadd_rn(dkey_inv(sel_v[s]), dkey_inv(sel_minr[s])));
    else if (n == 1)
        sp = dkey_inv(sel_minr[s]);
    else
        sp = __dmul_rn(0.5, __dadd_rn(lo[3 * g + ax], hi[3 * g + ax]));
    plane[g] = sp;
    const int64_t a = 2 * g + 1, c = 2 * g + 2;
    for (int d = 0; d < 3; d++) {
        lo[3 * a + d] = lo[3 * g + d];
        hi[3 * a + d] = hi[3 * g + d];
        lo[3 * c + d] = lo[3 * g + d];
        hi[3 * c + d] = hi[3 * g + d];
    }
    hi[3 * a + ax] = sp;
    lo[3 * c + ax] = sp;
    box_geometry(lo, hi, centre, radius, axis, a);
    box_geometry(lo, hi, centre, radius, axis, c);
}

// eta in [0,1): the plane s = eta * median plane + (1 - eta) * cell midpoint
// (Sec. 2.1.2); the left child takes the points strictly below it.
__global__ void k_eta_plane(int level, double eta, const int32_t *count, const int32_t *axis,
                            const double *lo, const double *hi, const uint64_t *sel_v,
                            const unsigned long long *sel_minr, unsigned long long *thr,
                            double *splane) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= (1 << level)) return;
    const int64_t g = ((int64_t)1 << level) - 1 + s;
    const int n = count[g], ax = axis[g];
    const double mid = __dmul_rn(0.5, __dadd_rn(lo[3 * g + ax], hi[3 * g + ax]));
    double sm = mid;
    if (eta > 0.0) {
        if (n >= 2)
            sm = __dmul_rn(0.5, __dadd_rn(dkey_inv(sel_v[s]), dkey_inv(sel_minr[s])));
        else if (n == 1)
            sm = dkey_inv(sel_v[s]);
    }
    const double sp = __dadd_rn(__dmul_rn(eta, sm), __dmul_rn(__dsub_rn(1.0, eta), mid));
    splane[s] = sp;
    thr[s] = dkey(sp);
}

// children of level `level` for the threshold split: cells cut at the plane,
// point ranges from the left counts; the largest child count for the host
__global__ void k_children_eta(int level, int32_t *begin, int32_t *count, const int32_t *ksplit,
                               const double *splane, double *lo, double *hi, double *centre,
                               double *radius, int32_t *axis, double *plane, int *maxcount) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= (1 << level)) return;
    const int64_t g = ((int64_t)1 << level) - 1 + s;
    const int n = count[g], ax = axis[g], k = ksplit[s], b = begin[g];
    const double sp = splane[s];
    plane[g] = sp;
    const int64_t a = 2 * g + 1, c = 2 * g + 2;
    begin[a] = b;
    count[a] = k;
    begin[c] = b + k;
    count[c] = n - k;
    for (int d = 0; d < 3; d++) {
        lo[3 * a + d] = lo[3 * g + d];
        hi[3 * a + d] = hi[3 * g + d];
        lo[3 * c + d] = lo[3 * g + d];
        hi[3 * c + d] = hi[3 * g + d];
    }
    hi[3 * a + ax] = sp;
    lo[3 * c + ax] = sp;
    box_geometry(lo, hi, centre, radius, axis, a);
    box_geometry(lo, hi, centre, radius, axis, c);
    atomicMax(maxcount, max(k, n - k));
}

}  // namespace

// Builds the tree: points (device, n x 3, dtype) -> leaf-order SoA positions,
// permutation, and all box cells/geometry. Box begin/count are host-computed
// (they depend on n and the level only) and already on the device.
cudaError_t tree_build(Plan &P, const void *pts, int dtype) {
    const int64_t n = P.n;
    cudaStream_t st = P.stream;
    const size_t nb = (size_t)n;
    // ping-pong buffers
    double *x2 = (double *)dalloc(P, nb * 8), *y2 = (double *)dalloc(P, nb * 8),
           *z2 = (double *)dalloc(P, nb * 8);
    int32_t *i2 = (int32_t *)dalloc(P, nb * 4);
    const int maxseg = 1 << (P.B > 0 ? P.B - 1 : 0);
    uint64_t *sel_v = (uint64_t *)dalloc(P, (size_t)maxseg * 8);
    uint64_t *sel_prefix = (uint64_t *)dalloc(P, (size_t)maxseg * 8);
    unsigned long long *sel_minr = (unsigned long long *)dalloc(P, (size_t)maxseg * 8);
    unsigned *sel_rrem = (unsigned *)dalloc(P, (size_t)maxseg * 4);
    unsigned *arrived = (unsigned *)dalloc(P, (size_t)maxseg * 4);  // per-box chunk arrivals
    unsigned *sel_found = (unsigned *)dalloc(P, (size_t)maxseg * 4);  // per-box early finish of the select
    unsigned long long *bbox = (unsigned long long *)dalloc(P, 64);
    if (!x2 || !y2 || !z2 || !i2 || !sel_v || !sel_prefix || !sel_minr || !sel_rrem || !arrived || !sel_found ||
        !bbox)
        return cudaErrorMemoryAllocation;
    cudaMemsetAsync(arrived, 0, (size_t)maxseg * 4, st);

    unsigned long long init[6] = {~0ull, ~0ull, ~0ull, 0ull, 0ull, 0ull};
    cudaMemcpyAsync(bbox, init, sizeof(init), cudaMemcpyHostToDevice, st);
    const int pgrid = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)sm_count() * 8);
    if (dtype == FMM_F64)
        FMM_LAUNCH(k_prepare<double>, pgrid, kThreads, 0, st, (const double *)pts, n, P.x, P.y, P.z,
                                                      P.perm, bbox, P.d_err);
    else
        FMM_LAUNCH(k_prepare<float>, pgrid, kThreads, 0, st, (const float *)pts, n, P.x, P.y, P.z,
                                                     P.perm, bbox, P.d_err);
    FMM_LAUNCH(k_root, 1, 32, 0, st, bbox, P.root, P.lo, P.hi, P.centre, P.radius, P.axis, P.d_err);

    double *xa = P.x, *ya = P.y, *za = P.z, *xb = x2, *yb = y2, *zb = z2;
    int32_t *ia = P.perm, *ib = i2;
    unsigned *ghist = nullptr, *chunk_lt = nullptr, *chunk_eq = nullptr, *eq_off = nullptr,
             *left_off = nullptr;
    size_t chunk_alloc = 0, ghist_alloc = 0;
    // eta < 1: data-dependent child sizes; the plane, the left counts and the
    // largest child count (read back per level to pick the regime) live here
    const bool eta_mode = P.eta < 1.0;
    const bool need_median = !eta_mode || P.eta > 0.0;
    unsigned long long *thr = nullptr;
    double *splane = nullptr;
    int32_t *ksplit = nullptr;
    int *dmax = nullptr;
    if (eta_mode) {
        thr = (unsigned long long *)dalloc(P, (size_t)maxseg * 8);
        splane = (double *)dalloc(P, (size_t)maxseg * 8);
        ksplit = (int32_t *)dalloc(P, (size_t)maxseg * 4);
        dmax = (int *)dalloc(P, 16);
        if (!thr || !splane || !ksplit || !dmax) return cudaErrorMemoryAllocation;
    }
    int64_t maxn = n;
    for (int l = 0; l < P.B; l++) {
        const int S = 1 << l;
        const unsigned sg = (unsigned)((S + 127) / 128);
        if (!eta_mode) maxn = (n + S - 1) / S;
        if (maxn <= kSmallCap) {
            if (need_median)
                FMM_LAUNCH(k_split_small, S, kThreads, 0, st, l, xa, ya, za, ia, xb, yb, zb, ib, P.begin,
                                                      P.count, P.axis, sel_v, sel_minr, P.d_err,
                                                      (const unsigned long long *)nullptr, (int32_t *)nullptr);
            if (eta_mode) {
                FMM_LAUNCH(k_eta_plane, sg, 128, 0, st, l, P.eta, P.count, P.axis, P.lo, P.hi, sel_v,
                                                       sel_minr, thr, splane);
                FMM_LAUNCH(k_split_small, S, kThreads, 0, st, l, xa, ya, za, ia, xb, yb, zb, ib, P.begin,
                                                      P.count, P.axis, sel_v, sel_minr, P.d_err,
                                                      (const unsigned long long *)thr, ksplit);
            }
        } else {
            const int nch = (int)((maxn + kChunk - 1) / kChunk);
            const size_t need_c = (size_t)S * nch * 4, need_h = (size_t)S * 256 * 4;
            if (need_c > chunk_alloc) {
                if (chunk_alloc) {
                    dfree(P, chunk_lt, chunk_alloc);
                    dfree(P, chunk_eq, chunk_alloc);
                    dfree(P, eq_off, chunk_alloc);
                    dfree(P, left_off, chunk_alloc);
                }
                chunk_alloc = need_c;
                chunk_lt = (unsigned *)dalloc(P, need_c);
                chunk_eq = (unsigned *)dalloc(P, need_c);
                eq_off = (unsigned *)dalloc(P, need_c);
                left_off = (unsigned *)dalloc(P, need_c);
                if (!chunk_lt || !chunk_eq || !eq_off || !left_off) return cudaErrorMemoryAllocation;
            }
            if (need_h > ghist_alloc) {
                if (ghist_alloc) dfree(P, ghist, ghist_alloc);
                ghist_alloc = need_h;
                ghist = (unsigned *)dalloc(P, need_h);
                if (!ghist) return cudaErrorMemoryAllocation;
            }
            const dim3 grid(S, nch);  // boxes on x (up to 2^31 - 1), chunks on y
            if (need_median) {
                FMM_LAUNCH(k_sel_init, S, 256, 0, st, l, P.count, sel_prefix, sel_rrem, sel_minr, ghist,
                           sel_found);
                for (int pass = 0; pass < 8; pass++)
                    FMM_LAUNCH(k_sel_hist, grid, kThreads, 0, st, l, pass, xa, ya, za, P.begin, P.count,
                                                          P.axis, sel_prefix, sel_rrem, ghist, arrived, sel_found);
                FMM_LAUNCH(k_sel_count, grid, kThreads, 0, st, l, nch, xa, ya, za, P.begin, P.count, P.axis,
                                                       sel_prefix, chunk_lt, chunk_eq, sel_minr,
                                                       (const unsigned long long *)nullptr);
                FMM_LAUNCH(k_sel_offsets, sg, 128, 0, st, l, nch, P.count, chunk_lt, chunk_eq, sel_prefix,
                                                       sel_rrem, eq_off, left_off, sel_minr, sel_v,
                                                       (const unsigned long long *)nullptr, (int32_t *)nullptr);
            }
            if (!eta_mode) {
                FMM_LAUNCH(k_sel_scatter, grid, kThreads, 0, st, l, nch, xa, ya, za, ia, xb, yb, zb, ib,
                                                         P.begin, P.count, P.axis, sel_prefix, sel_rrem, eq_off,
                                                         left_off, P.d_err, (const unsigned long long *)nullptr,
                                                         (const int32_t *)nullptr);
            } else {
                FMM_LAUNCH(k_eta_plane, sg, 128, 0, st, l, P.eta, P.count, P.axis, P.lo, P.hi, sel_v,
                                                       sel_minr, thr, splane);
                FMM_LAUNCH(k_sel_count, grid, kThreads, 0, st, l, nch, xa, ya, za, P.begin, P.count, P.axis,
                                                       sel_prefix, chunk_lt, chunk_eq, sel_minr,
                                                       (const unsigned long long *)thr);
                FMM_LAUNCH(k_sel_offsets, sg, 128, 0, st, l, nch, P.count, chunk_lt, chunk_eq, sel_prefix,
                                                       sel_rrem, eq_off, left_off, sel_minr, sel_v,
                                                       (const unsigned long long *)thr, ksplit);
                FMM_LAUNCH(k_sel_scatter, grid, kThreads, 0, st, l, nch, xa, ya, za, ia, xb, yb, zb, ib,
                                                         P.begin, P.count, P.axis, sel_prefix, sel_rrem, eq_off,
                                                         left_off, P.d_err, (const unsigned long long *)thr,
                                                         (const int32_t *)ksplit);
            }
        }
        if (!eta_mode) {
            FMM_LAUNCH(k_children, sg, 128, 0, st, l, P.count, sel_v, sel_minr, P.lo, P.hi, P.centre,
                                                        P.radius, P.axis, P.plane);
        } else {
            cudaMemsetAsync(dmax, 0, 4, st);
            FMM_LAUNCH(k_children_eta, sg, 128, 0, st, l, P.begin, P.count, ksplit, splane, P.lo, P.hi,
                                                            P.centre, P.radius, P.axis, P.plane, dmax);
            int hmax = 0;
            cudaMemcpyAsync(&hmax, dmax, 4, cudaMemcpyDeviceToHost, st);
            const cudaError_t es = cudaStreamSynchronize(st);
            if (es != cudaSuccess) return es;
            maxn = hmax;
        }
        std::swap(xa, xb);
        std::swap(ya, yb);
        std::swap(za, zb);
        std::swap(ia, ib);
    }
    cudaError_t e = cudaGetLastError();
    // leave the final order in the plan's primary buffers
    if (xa != P.x) {
        cudaMemcpyAsync(P.x, xa, nb * 8, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(P.y, ya, nb * 8, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(P.z, za, nb * 8, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(P.perm, ia, nb * 4, cudaMemcpyDeviceToDevice, st);
    }
    if (chunk_alloc) {
        dfree(P, chunk_lt, chunk_alloc);
        dfree(P, chunk_eq, chunk_alloc);
        dfree(P, eq_off, chunk_alloc);
        dfree(P, left_off, chunk_alloc);
    }
    if (ghist_alloc) dfree(P, ghist, ghist_alloc);
    dfree(P, x2, nb * 8);
    dfree(P, y2, nb * 8);
    dfree(P, z2, nb * 8);
    dfree(P, i2, nb * 4);
    dfree(P, sel_v, (size_t)maxseg * 8);
    dfree(P, sel_prefix, (size_t)maxseg * 8);
    dfree(P, sel_minr, (size_t)maxseg * 8);
    dfree(P, sel_rrem, (size_t)maxseg * 4);
    dfree(P, arrived, (size_t)maxseg * 4);
    dfree(P, bbox, 64);
    if (eta_mode) {
        dfree(P, thr, (size_t)maxseg * 8);
        dfree(P, splane, (size_t)maxseg * 8);
        dfree(P, ksplit, (size_t)maxseg * 4);
        dfree(P, dmax, 16);
    }
    return e;
}

// ---------------------------------------------------------------------------
// Tight box geometry (FMM_FLAG_TIGHT): the expansion centre and radius of a
// box from the bounding box of its own points, the radius floored at 2^-10
// of the cell radius (a box of one point keeps a positive size; an empty box
// keeps its cell midpoint). The cells, which decide the splits, are kept.
// Min and max are exact, so any reduction order gives the oracle's bits.
// ---------------------------------------------------------------------------
namespace {

// One warp per leaf reduces its points; the lane-0 thread then walks up the
// tree: a parent is formed by the second of its two children to arrive
// (an arrival counter per internal box), so no thread ever waits.
__global__ void k_tight_boxes(int B, const double *__restrict__ x, const double *__restrict__ y,
                              const double *__restrict__ z, const int32_t *__restrict__ begin,
                              const int32_t *__restrict__ count, double *tlo, double *thi,
                              unsigned *arrive) {
    const int64_t nl = (int64_t)1 << B;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double *src[3] = {x, y, z};
    // min and max on the order-preserving integer keys of the coordinates
    // (exact, and equal to fmin / fmax here: no NaN, -0 canonicalised to +0),
    // off the narrow FP64 pipe
    for (int64_t j = warp; j < nl; j += nwarps) {
        int64_t g = nl - 1 + j;
        const int b = begin[g], n = count[g];
        uint64_t lo[3], hi[3];
        for (int a = 0; a < 3; a++) {
            uint64_t l = 0xfff0000000000000ull, h = 0x000fffffffffffffull;  // dkey(+inf), dkey(-inf)
            for (int i = lane; i < n; i += 32) {
                const uint64_t v = dkey(src[a][b + i]);
                l = min(l, v);
                h = max(h, v);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                l = min(l, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)l, o));
                h = max(h, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)h, o));
            }
            lo[a] = l;
            hi[a] = h;
        }
        if (lane == 0) {
            for (int a = 0; a < 3; a++) {
                tlo[3 * g + a] = dkey_inv(lo[a]);
                thi[3 * g + a] = dkey_inv(hi[a]);
            }
            while (g > 0) {
                __threadfence();
                const int64_t par = (g - 1) >> 1;
                if (atomicAdd(&arrive[par], 1u) == 0) break;  // the sibling forms the parent
                __threadfence();
                const int64_t c0 = 2 * par + 1, c1 = c0 + 1;
                for (int a = 0; a < 3; a++) {
                    tlo[3 * par + a] = dkey_inv(min(dkey(__ldcg(tlo + 3 * c0 + a)), dkey(__ldcg(tlo + 3 * c1 + a))));
                    thi[3 * par + a] = dkey_inv(max(dkey(__ldcg(thi + 3 * c0 + a)), dkey(__ldcg(thi + 3 * c1 + a))));
                }
                g = par;
            }
        }
    }
}

// centre = 0.5 (lo + hi), radius = max(0.5 sqrt((ex^2 + ey^2) + ez^2), 2^-10 r_cell)
// in the oracle's operation order without contraction; empty boxes keep the
// cell midpoint and take the floor, and their point box becomes that point.
__global__ void k_tight_geometry(int64_t nbox, const int32_t *__restrict__ count, double *__restrict__ centre,
                                 double *__restrict__ radius, double *__restrict__ tlo,
                                 double *__restrict__ thi) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= nbox) return;
    const double floor_r = __dmul_rn(radius[g], 0x1p-10);
    if (count[g] == 0) {
        radius[g] = floor_r;
        for (int a = 0; a < 3; a++) tlo[3 * g + a] = thi[3 * g + a] = centre[3 * g + a];
        return;
    }
    double e[3];
    for (int a = 0; a < 3; a++) {
        const double l = tlo[3 * g + a], h = thi[3 * g + a];
        e[a] = __dsub_rn(h, l);
        centre[3 * g + a] = __dmul_rn(0.5, __dadd_rn(l, h));
    }
    const double s = __dadd_rn(__dadd_rn(__dmul_rn(e[0], e[0]), __dmul_rn(e[1], e[1])), __dmul_rn(e[2], e[2]));
    const double r = __dmul_rn(0.5, __dsqrt_rn(s));
    radius[g] = r > floor_r ? r : floor_r;
}

}  // namespace

cudaError_t tight_geometry(Plan &P) {
    cudaStream_t st = P.stream;
    const size_t nb = (size_t)P.nbox;
    P.tlo = (double *)dalloc(P, nb * 24);
    P.thi = (double *)dalloc(P, nb * 24);
    unsigned *arrive = (unsigned *)dalloc(P, nb * 4);
    if (!P.tlo || !P.thi || !arrive) return cudaErrorMemoryAllocation;
    cudaMemsetAsync(arrive, 0, nb * 4, st);
    const int64_t warps = P.nleaf;
    const unsigned grid = (unsigned)std::min<int64_t>((warps * 32 + 255) / 256, (int64_t)sm_count() * 16);
    FMM_LAUNCH(k_tight_boxes, grid, 256, 0, st, P.B, P.x, P.y, P.z, P.begin, P.count, P.tlo, P.thi, arrive);
    FMM_LAUNCH(k_tight_geometry, (unsigned)((nb + 255) / 256), 256, 0, st, P.nbox, P.count, P.centre, P.radius,
               P.tlo, P.thi);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free ORB leaf order for small point sets (fmm_orb_order_noalloc).
//
// For callers that cannot allocate device memory (host applications that
// own all device memory, loops that cannot wait on an allocator): the small-regime
// split kernels above run with every scratch buffer carved out of one static
// device array. Up to FMM_NOALLOC_MAX_POINTS points every level is in the
// one-CTA regime, so no chunk counters or histograms are needed.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNaMaxN = FMM_NOALLOC_MAX_POINTS;
constexpr int kNaMaxBoxes = (2 << FMM_NOALLOC_MAX_LEVELS) - 1;
constexpr int kNaMaxSeg = 1 << (FMM_NOALLOC_MAX_LEVELS - 1);
constexpr size_t na_round(size_t b) { return (b + 255) / 256 * 256; }
// byte offsets of the scratch buffers inside the static array
constexpr size_t kNaPos = 0;                                        // 6 x n doubles (2 copies of x|y|z)
constexpr size_t kNaIdx = kNaPos + na_round(6ull * kNaMaxN * 8);    // 2 x n int32
constexpr size_t kNaBox = kNaIdx + na_round(2ull * kNaMaxN * 4);    // begin|count|axis int32
constexpr size_t kNaGeo = kNaBox + na_round(3ull * kNaMaxBoxes * 4);  // lo|hi|centre (x3) radius|plane
constexpr size_t kNaSel = kNaGeo + na_round(11ull * kNaMaxBoxes * 8); // sel_v|sel_minr
constexpr size_t kNaMisc = kNaSel + na_round(2ull * kNaMaxSeg * 8);  // bbox[6] u64, err
constexpr size_t kNaEnd = kNaMisc + 256;
static_assert(kNaEnd <= FMM_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the declared size");

}  // namespace

// The scratch itself: file scope, one per device that loads the library.
static __device__ __align__(256) unsigned char g_orb_scratch[FMM_NOALLOC_SCRATCH_BYTES];

namespace {

// Resets what must start cleared (bounding box, error word, plane values) and
// writes the boxes' point ranges, which depend on n and the level only.
__global__ void k_noalloc_init(int n, int levels, int32_t *begin, int32_t *count,
                               unsigned long long *bbox, int *err, double *plane) {
    const int nb = (2 << levels) - 1;
    for (int g = threadIdx.x; g < nb; g += blockDim.x) plane[g] = 0.0;
    if (threadIdx.x == 0) {
        for (int a = 0; a < 3; a++) {
            bbox[a] = ~0ull;
            bbox[3 + a] = 0ull;
        }
        *err = 0;
        begin[0] = 0;
        count[0] = n;
        for (int g = 0; g < nb - (1 << levels); g++) {
            const int k = count[g] / 2;
            begin[2 * g + 1] = begin[g];
            count[2 * g + 1] = k;
            begin[2 * g + 2] = begin[g] + k;
            count[2 * g + 2] = count[g] - k;
        }
    }
}

unsigned char *g_na_addr[64] = {};
std::atomic<int> g_na_lock{0};

// Device address of g_orb_scratch on the current device (looked up once).
cudaError_t noalloc_scratch(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    while (g_na_lock.exchange(1, std::memory_order_acquire)) {
    }
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_orb_scratch);
        if (e == cudaSuccess) g_na_addr[dev] = (unsigned char *)p;
    }
    *out = g_na_addr[dev];
    g_na_lock.store(0, std::memory_order_release);
    return e;
}

}  // namespace

namespace {
// per box: centre split hi + lo in float (hi.xyz, lo.xyz) and its radius (hi.w)
__global__ void k_box_cf(int64_t nbox, const double *__restrict__ centre, const double *__restrict__ radius,
                         float4 *__restrict__ cf) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nbox; g += (int64_t)gridDim.x * blockDim.x) {
        float h[3], l[3];
        for (int d = 0; d < 3; d++) {
            const double c = centre[3 * g + d];
            h[d] = (float)c;
            l[d] = (float)(c - (double)h[d]);
        }
        cf[2 * g] = make_float4(h[0], h[1], h[2], (float)radius[g]);
        cf[2 * g + 1] = make_float4(l[0], l[1], l[2], 0.f);
    }
}
}  // namespace

void box_centres_f(Plan &P) {
    FMM_LAUNCH(k_box_cf, (unsigned)std::min<int64_t>((P.nbox + 255) / 256, (int64_t)sm_count() * 8), 256, 0,
               P.stream, P.nbox, P.centre, P.radius, P.box_cf);
}

}  // namespace fmm

extern "C" int fmm_orb_order_noalloc(const void *points, int64_t n, int dtype, int levels,
                                     int32_t *perm, void *stream) {
    using namespace fmm;
    if (!points || !perm || n < 1 || n > kNaMaxN || levels < 0 ||
        levels > FMM_NOALLOC_MAX_LEVELS || (dtype != FMM_F64 && dtype != FMM_F32))
        return FMM_EINVAL;
    if (ptr_kind(points) != 1 || ptr_kind(perm) != 1) return FMM_EINVAL;
    unsigned char *s = nullptr;
    cudaError_t e = noalloc_scratch(&s);
    if (e != cudaSuccess) return cuda_status(e);
    cudaStream_t st = (cudaStream_t)stream;
    double *pos = (double *)(s + kNaPos);
    double *xa = pos, *ya = pos + kNaMaxN, *za = pos + 2 * kNaMaxN;
    double *xb = pos + 3 * kNaMaxN, *yb = pos + 4 * kNaMaxN, *zb = pos + 5 * kNaMaxN;
    int32_t *ia = (int32_t *)(s + kNaIdx), *ib = ia + kNaMaxN;
    int32_t *begin = (int32_t *)(s + kNaBox), *count = begin + kNaMaxBoxes,
            *axis = begin + 2 * kNaMaxBoxes;
    double *geo = (double *)(s + kNaGeo);
    double *lo = geo, *hi = geo + 3 * kNaMaxBoxes, *centre = geo + 6 * kNaMaxBoxes;
    double *radius = geo + 9 * kNaMaxBoxes, *plane = geo + 10 * kNaMaxBoxes;
    uint64_t *sel_v = (uint64_t *)(s + kNaSel);
    unsigned long long *sel_minr = (unsigned long long *)(s + kNaSel) + kNaMaxSeg;
    unsigned long long *bbox = (unsigned long long *)(s + kNaMisc);
    int *err = (int *)(s + kNaMisc + 64);

    FMM_LAUNCH(k_noalloc_init, 1, 256, 0, st, (int)n, levels, begin, count, bbox, err, plane);
    const int pgrid = (int)((n + kThreads - 1) / kThreads);
    if (dtype == FMM_F64)
        FMM_LAUNCH(k_prepare<double>, pgrid, kThreads, 0, st, (const double *)points, n, xa, ya, za, ia,
                   bbox, err);
    else
        FMM_LAUNCH(k_prepare<float>, pgrid, kThreads, 0, st, (const float *)points, n, xa, ya, za, ia,
                   bbox, err);
    FMM_LAUNCH(k_root, 1, 32, 0, st, bbox, RootCell{}, lo, hi, centre, radius, axis, err);
    for (int l = 0; l < levels; l++) {
        const int S = 1 << l;
        FMM_LAUNCH(k_split_small, S, kThreads, 0, st, l, xa, ya, za, ia, xb, yb, zb, ib, begin, count,
                   axis, sel_v, sel_minr, err, (const unsigned long long *)nullptr, (int32_t *)nullptr);
        FMM_LAUNCH(k_children, (S + 127) / 128, 128, 0, st, l, count, sel_v, sel_minr, lo, hi, centre,
                   radius, axis, plane);
        std::swap(xa, xb);
        std::swap(ya, yb);
        std::swap(za, zb);
        std::swap(ia, ib);
    }
    e = cudaMemcpyAsync(perm, ia, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    if (herr & 1) return FMM_ENONFINITE;
    return herr ? FMM_EINTERNAL : FMM_OK;
}
