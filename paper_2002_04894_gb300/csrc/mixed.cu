// Mixed-precision leaf stages (FMM_PREC_MIXED): P2M, L2P and P2P in single
// precision, with the box geometry, the theta-test, M2M and L2L left in double
// precision and the multipole/local coefficients stored in double as before.
//
// Conditioning. Every point is kept as its offset a = x - c from its leaf
// centre, split into a float pair hi + lo (hi = float(a), lo = float(a - hi)).
// In P2P the source offsets are re-expressed relative to the target leaf's
// centre with an error-free float TwoSum, so the difference of a close pair is
// taken between two nearly equal hi parts, which is exact (Sterbenz), and
// close pairs keep full relative precision. Per-target sums are plain float
// over runs of 64 sources and Kahan-compensated across runs (the rounding of
// a 64-term sum stays near the float unit roundoff while the compensation
// costs a fraction of an instruction per pair). P2M and L2P evaluate on
// scaled offsets a / s (s = 2^e within a factor 2 below the leaf's radius, so
// |a / s| < 2) with scaled coefficients M_n / s^n and L_n s^n; the M2L reads
// M_n / r^n and forms r^k L_k (r the box radius). Every float value stays
// O(1) whatever the box size.

#include <algorithm>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

// 1/k for k = 0..FMM_MAX_P^2 (0 at k = 0): the harmonic recurrences divide by
// (n - m)(n + m) = n^2 - m^2 once per term; the reciprocal of that integer,
// correctly rounded, is read here (warp-uniform index, constant cache)
struct InvTable {
    float v[FMM_MAX_P * FMM_MAX_P + 1];
};
constexpr InvTable make_inv_table() {
    InvTable t{};
    for (int k = 1; k <= FMM_MAX_P * FMM_MAX_P; k++) t.v[k] = 1.0f / (float)k;
    return t;
}
__constant__ InvTable c_inv = make_inv_table();

constexpr int kThreads = 128;

__device__ __forceinline__ float2 fcmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// The leaf's scale s = 2^e with s <= r < 2 s (r its radius; 1 for r = 0):
// offsets are taken over s (|x / s| < 2 in the box), and the coefficients
// scale by s^n, a power of two formed exactly without a power loop in double
__device__ __forceinline__ int box_scale_exp(double r) { return r > 0.0 ? max(-48, min(48, ilogb(r))) : 0; }

// offsets from the leaf centre, split hi/lo
__global__ void k_leaf_offsets(int B, int64_t n, const double *__restrict__ x,
                               const double *__restrict__ y, const double *__restrict__ z,
                               const int32_t *__restrict__ begin, const int32_t *__restrict__ count,
                               const double *__restrict__ centre, float *__restrict__ hl) {
    const int64_t g = ((int64_t)1 << B) - 1 + blockIdx.x;
    const int b = begin[g], cnt = count[g];
    const double c[3] = {centre[3 * g], centre[3 * g + 1], centre[3 * g + 2]};
    const double *src[3] = {x, y, z};
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        for (int a = 0; a < 3; a++) {
            const double d = src[a][b + i] - c[a];
            const float h = (float)d;
            hl[a * n + b + i] = h;
            hl[(3 + a) * n + b + i] = (float)(d - (double)h);
        }
    }
}

template <typename T>
__global__ void k_gather_qf(const T *__restrict__ qin, const int32_t *__restrict__ perm,
                            float *__restrict__ q, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        q[i] = (float)qin[perm[i]];
}

// P2M on scaled offsets a / s (s = 2^e, the power of two within a factor
// 2 below the leaf's radius), one warp per leaf: each lane carries kP2MSlots
// points, and two warp sums per coefficient (slots 0-1 and 2-3, 64 points
// each) cover a batch of 128; the two sums stay apart in float in shared
// memory and are combined in double, so each float sum is no deeper than
// a 64-term tree. The leaf's multipole is stored unscaled in double
// (M_n^m = s^n Mhat_n^m, s^n exact).
constexpr int kP2MSlots = 4;
__device__ __forceinline__ void p2m_f32_body(int B, int p, int64_t n, const float *__restrict__ hl,
                                             const float *__restrict__ q, const int32_t *__restrict__ begin,
                                             const int32_t *__restrict__ count, const double *__restrict__ radius,
                                             double2 *__restrict__ M, int64_t leaf) {
    extern __shared__ float2 accf[];  // [2][nc]
    const int nc = ncoef(p);
    const int64_t g = ((int64_t)1 << B) - 1 + leaf;
    const int b = begin[g], cnt = count[g];
    const int lane = threadIdx.x;
    const int es = box_scale_exp(radius[g]);
    const float rinv = (float)pow2i(-es);
    for (int c = lane; c < 2 * nc; c += 32) accf[c] = make_float2(0.f, 0.f);
    __syncwarp();
    for (int base = 0; base < cnt; base += 32 * kP2MSlots) {
        float sx[kP2MSlots], sy[kP2MSlots], sz[kP2MSlots], r2[kP2MSlots], qi[kP2MSlots];
        float2 mm[kP2MSlots];
#pragma unroll
        for (int r = 0; r < kP2MSlots; r++) {
            const int i = base + 32 * r + lane;
            const bool valid = i < cnt;
            sx[r] = valid ? (hl[b + i] + hl[3 * n + b + i]) * rinv : 0.f;
            sy[r] = valid ? (hl[n + b + i] + hl[4 * n + b + i]) * rinv : 0.f;
            sz[r] = valid ? (hl[2 * n + b + i] + hl[5 * n + b + i]) * rinv : 0.f;
            qi[r] = valid ? q[b + i] : 0.f;
            r2[r] = sx[r] * sx[r] + sy[r] * sy[r] + sz[r] * sz[r];
            mm[r] = make_float2(1.f, 0.f);
        }
        for (int m = 0; m <= p; m++) {
            float2 cur[kP2MSlots], prev[kP2MSlots];
#pragma unroll
            for (int r = 0; r < kP2MSlots; r++) {
                if (m > 0) {
                    mm[r] = fcmul(mm[r], make_float2(sx[r], sy[r]));
                    const float s = 0.5f / m;
                    mm[r] = make_float2(mm[r].x * s, mm[r].y * s);
                }
                cur[r] = mm[r];
                prev[r] = make_float2(0.f, 0.f);
            }
            for (int nn = m; nn <= p; nn++) {
                float vr[2] = {0.f, 0.f}, vi[2] = {0.f, 0.f};
#pragma unroll
                for (int r = 0; r < kP2MSlots; r++) {
                    if (nn > m) {
                        float2 nxt;
                        if (nn == m + 1) {
                            nxt = make_float2(cur[r].x * sz[r], cur[r].y * sz[r]);
                        } else {
                            const float s = c_inv.v[nn * nn - m * m];  // 1 / ((n - m)(n + m))
                            const float a = (2 * nn - 1) * sz[r];
                            nxt = make_float2((a * cur[r].x - r2[r] * prev[r].x) * s,
                                              (a * cur[r].y - r2[r] * prev[r].y) * s);
                        }
                        prev[r] = cur[r];
                        cur[r] = nxt;
                    }
                    const float sg = (m & 1) ? -qi[r] : qi[r];
                    vr[r >> 1] = fmaf(sg, cur[r].x, vr[r >> 1]);
                    vi[r >> 1] = fmaf(-sg, cur[r].y, vi[r >> 1]);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        vr[h] += __shfl_xor_sync(0xffffffffu, vr[h], o);
                        vi[h] += __shfl_xor_sync(0xffffffffu, vi[h], o);
                    }
                }
                if (lane == 0) {
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const float2 a = accf[h * nc + tri(nn, m)];
                        accf[h * nc + tri(nn, m)] = make_float2(a.x + vr[h], a.y + vi[h]);
                    }
                }
            }
        }
    }
    __syncwarp();
    for (int c = lane; c < nc; c += 32) {
        int nn = 0;
        while (tri(nn + 1, 0) <= c) nn++;
        const double s = pow2i(es * nn);
        M[g * nc + c] = make_double2(((double)accf[c].x + (double)accf[nc + c].x) * s,
                                     ((double)accf[c].y + (double)accf[nc + c].y) * s);
    }
}

__global__ void __launch_bounds__(32)
k_p2m_f32(int B, int p, int64_t n, const float *__restrict__ hl, const float *__restrict__ q,
          const int32_t *__restrict__ begin, const int32_t *__restrict__ count,
          const double *__restrict__ radius, double2 *__restrict__ M) {
    p2m_f32_body(B, p, n, hl, q, begin, count, radius, M, blockIdx.x);
}

// batched: one block per leaf of every system (block offsets per system)
__global__ void __launch_bounds__(32)
k_b_p2m_f32(const BatchSys *__restrict__ S, const int32_t *__restrict__ off, int nsys) {
    const int s = batch_sys_of(off, nsys, blockIdx.x);
    const BatchSys &y = S[s];
    p2m_f32_body(y.B, y.p, y.n, y.hl, y.qf, y.begin, y.count, y.radius, y.M, blockIdx.x - off[s]);
}

// L2P on scaled offsets: Lhat_k^l = s^k L_k^l (s = 2^e near the leaf's
// radius, s^k exact); phi = sum Lhat conj(Y(a/s)); E = -grad phi =
// (Re G1, Im G1, -G0) / s with the degree-1 shifted terms.
__device__ __forceinline__ void l2p_f32_body(int B, int p, int64_t n, const float *__restrict__ hl,
                                             const int32_t *__restrict__ begin, const int32_t *__restrict__ count,
                                             const double *__restrict__ radius, const double2 *__restrict__ L,
                                             float *__restrict__ far_phi, float *__restrict__ far_E, int64_t leaf) {
    extern __shared__ float2 Ls[];
    const int nc = ncoef(p);
    const int64_t g = ((int64_t)1 << B) - 1 + leaf;
    const int b = begin[g], cnt = count[g];
    const int es = box_scale_exp(radius[g]);
    for (int c = threadIdx.x; c < nc; c += kThreads) {
        int nn = 0;
        while (tri(nn + 1, 0) <= c) nn++;
        const double s = pow2i(es * nn);
        const double2 v = L[g * nc + c];
        Ls[c] = make_float2((float)(v.x * s), (float)(v.y * s));
    }
    __syncthreads();
    const float rinv = (float)pow2i(-es);
    for (int i = threadIdx.x; i < cnt; i += kThreads) {
        const float sx = (hl[b + i] + hl[3 * n + b + i]) * rinv;
        const float sy = (hl[n + b + i] + hl[4 * n + b + i]) * rinv;
        const float sz = (hl[2 * n + b + i] + hl[5 * n + b + i]) * rinv;
        const float r2 = sx * sx + sy * sy + sz * sz;
        float phi = 0.f, g0 = 0.f;
        float2 g1 = make_float2(0.f, 0.f);
        float2 mm = make_float2(1.f, 0.f);
        for (int m = 0; m <= p; m++) {
            if (m > 0) {
                mm = fcmul(mm, make_float2(sx, sy));
                const float s = 0.5f / m;
                mm = make_float2(mm.x * s, mm.y * s);
            }
            float2 cur = mm, prev = make_float2(0.f, 0.f);
            const float w = m == 0 ? 1.f : 2.f;
            for (int nn = m; nn <= p; nn++) {
                if (nn > m) {
                    float2 nxt;
                    if (nn == m + 1) {
                        nxt = make_float2(cur.x * sz, cur.y * sz);
                    } else {
                        const float s = c_inv.v[nn * nn - m * m];  // 1 / ((n - m)(n + m))
                        const float a = (2 * nn - 1) * sz;
                        nxt = make_float2((a * cur.x - r2 * prev.x) * s, (a * cur.y - r2 * prev.y) * s);
                    }
                    prev = cur;
                    cur = nxt;
                }
                const float2 Y = (m & 1) ? make_float2(-cur.x, -cur.y) : cur;
                const float2 Yc = make_float2(Y.x, -Y.y);
                phi += w * fcmul(Ls[tri(nn, m)], Yc).x;
                if (nn < p) {
                    g0 += w * fcmul(Ls[tri(nn + 1, m)], Yc).x;
                    const float2 a = fcmul(Ls[tri(nn + 1, m + 1)], Yc);
                    g1.x += a.x;
                    g1.y += a.y;
                    if (m >= 1) {
                        const float2 lc = Ls[tri(nn + 1, m - 1)];
                        const float2 t = fcmul(make_float2(lc.x, -lc.y), Y);
                        g1.x -= t.x;
                        g1.y -= t.y;
                    }
                }
            }
        }
        far_phi[b + i] = phi;
        far_E[b + i] = g1.x * rinv;
        far_E[n + b + i] = g1.y * rinv;
        far_E[2 * n + b + i] = -g0 * rinv;
    }
}

__global__ void __launch_bounds__(kThreads)
k_l2p_f32(int B, int p, int64_t n, const float *__restrict__ hl, const int32_t *__restrict__ begin,
          const int32_t *__restrict__ count, const double *__restrict__ radius,
          const double2 *__restrict__ L, float *__restrict__ far_phi, float *__restrict__ far_E) {
    l2p_f32_body(B, p, n, hl, begin, count, radius, L, far_phi, far_E, blockIdx.x);
}

__global__ void __launch_bounds__(kThreads)
k_b_l2p_f32(const BatchSys *__restrict__ S, const int32_t *__restrict__ off, int nsys) {
    const int s = batch_sys_of(off, nsys, blockIdx.x);
    const BatchSys &y = S[s];
    l2p_f32_body(y.B, y.p, y.n, y.hl, y.begin, y.count, y.radius, y.L, y.far_phi, y.far_E, blockIdx.x - off[s]);
}

__device__ __forceinline__ void kahan(float &s, float &c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// exact float sum a + b = s + e (Knuth TwoSum)
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
    const float s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}

// per leaf, in float: centre hi (xyz) + radius | centre lo | half extents
__global__ void k_leaf_geo(int B, const double *__restrict__ lo, const double *__restrict__ hi,
                           const double *__restrict__ centre, const double *__restrict__ radius,
                           float4 *__restrict__ geo) {
    const int64_t nl = (int64_t)1 << B;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= nl) return;
    const int64_t g = nl - 1 + j;
    float h[3], l[3], e[3];
    for (int a = 0; a < 3; a++) {
        const double c = centre[3 * g + a];
        h[a] = (float)c;
        l[a] = (float)(c - (double)h[a]);
        e[a] = (float)(0.5 * (hi[3 * g + a] - lo[3 * g + a]));
    }
    geo[3 * j] = make_float4(h[0], h[1], h[2], (float)radius[g]);
    geo[3 * j + 1] = make_float4(l[0], l[1], l[2], 0.f);
    geo[3 * j + 2] = make_float4(e[0], e[1], e[2], 0.f);
}

constexpr int kLeafChunk = 128;
constexpr float kFarGap = 0.1f;   // far: cell gap >= kFarGap (r_t + r_s)
constexpr float kPadFar = 1.0e18f;  // padding source: zero charge, far away
constexpr int kRun = 64;  // sources summed in float before the compensated add

__device__ __forceinline__ float rcp_approx(float x) {  // reciprocal on the XU pipe (~1 ulp)
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// 1/sqrt on the XU pipe, denormal inputs flushed: rsqrtf's handling of
// denormal arguments costs extra instructions per call, and a far pair's r^2
// (at least (0.1 (r_t + r_s))^2) is never denormal
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// One target against two sources at once, in packed float2 arithmetic. The
// sources of a pair are staged as A = (-x0, -x1, -y0, -y1) and
// B = (-z0, -z1, q0, q1), offsets from the target leaf's centre; the sums run
// separately over even and odd sources.
// far (cells apart): single-float offsets
__device__ __forceinline__ void far_pair2(float2 X, float2 Y, float2 Z, const float4 A, const float4 B,
                                          float2 *a) {
    const float2 dx = add2(X, make_float2(A.x, A.y));
    const float2 dy = add2(Y, make_float2(A.z, A.w));
    const float2 dz = add2(Z, make_float2(B.x, B.y));
    const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
    const float2 rinv = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
    const float2 rinv2 = mul2(rinv, rinv);  // one packed product: fewer issue slots than two XU reciprocals
    const float2 qr = mul2(make_float2(B.z, B.w), rinv);
    const float2 qr3 = mul2(qr, rinv2);
    a[0] = add2(a[0], qr);
    a[1] = fma2(qr3, dx, a[1]);
    a[2] = fma2(qr3, dy, a[2]);
    a[3] = fma2(qr3, dz, a[3]);
}

// near (touching cells): split hi/lo offsets (lo parts staged as
// C = (-xl0, -xl1, -yl0, -yl1), D = (-zl0, -zl1, ., .)), coincident points
// skipped
__device__ __forceinline__ void near_pair2(float2 X, float2 Y, float2 Z, float2 XL, float2 YL, float2 ZL,
                                           const float4 A, const float4 B, const float4 C, const float4 D,
                                           float2 *a) {
    const float2 dx = add2(add2(X, make_float2(A.x, A.y)), add2(XL, make_float2(C.x, C.y)));
    const float2 dy = add2(add2(Y, make_float2(A.z, A.w)), add2(YL, make_float2(C.z, C.w)));
    const float2 dz = add2(add2(Z, make_float2(B.x, B.y)), add2(ZL, make_float2(D.x, D.y)));
    const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
    const float2 rinv = make_float2(r2.x > 0.f ? rsqrtf(r2.x) : 0.f, r2.y > 0.f ? rsqrtf(r2.y) : 0.f);
    const float2 rinv2 = make_float2(r2.x > 0.f ? rcp_approx(r2.x) : 0.f, r2.y > 0.f ? rcp_approx(r2.y) : 0.f);
    const float2 qr = mul2(make_float2(B.z, B.w), rinv);
    const float2 qr3 = mul2(qr, rinv2);
    a[0] = add2(a[0], qr);
    a[1] = fma2(qr3, dx, a[1]);
    a[2] = fma2(qr3, dy, a[2]);
    a[3] = fma2(qr3, dz, a[3]);
}

// exclusive prefix of v[0..len) in place (len <= kLeafChunk), the total at
// v[len]; block-wide (T threads), synchronised on return
template <int T>
__device__ __forceinline__ void block_excl_scan(int *v, int len, int *wsum) {
    constexpr int kPer = (kLeafChunk + T - 1) / T;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int k0 = tid * kPer;
    int loc[kPer], own = 0;
#pragma unroll
    for (int i = 0; i < kPer; i++) {
        loc[i] = k0 + i < len ? v[k0 + i] : 0;
        own += loc[i];
    }
    int inc = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int run = inc - own;
    for (int i = 0; i < w; i++) run += wsum[i];
#pragma unroll
    for (int i = 0; i < kPer; i++) {
        if (k0 + i < len) v[k0 + i] = run;
        run += loc[i];
    }
    if (tid == T - 1) v[len] = run;  // entries past len count zero
    __syncthreads();
}

// Near field in float. One CTA per work unit (a tile of up to T = 128 or 64
// targets of one leaf, by the plan's mean leaf size; heaviest units first),
// one target point per thread, two sources per step in packed float2
// arithmetic (FFMA2/FADD2/FMUL2). For
// every source leaf the offset between the two leaf centres is formed once,
// error-free (float TwoSum on the centres' hi/lo parts), together with a
// near/far flag: far when the gap g between the two cells is at least
// kFarGap (r_t + r_s). The float offsets then carry an absolute error of
// about 2u (r_t + r_s + |offset|), and since strongly connected leaves have
// |offset| < 3 max(r_t, r_s), every far pair's distance (>= g) is known to
// at worst ~100u relative (the closest far pairs only; ~75% of pairs sit at
// g >= 0.5 (r_t + r_s), known to ~20u): a single float per coordinate
// suffices, and no two points can coincide. Near leaves (touching or nearly
// touching cells, ~4% of the pairs on a Plummer sphere) keep the split hi/lo
// offsets, whose difference is exact for close pairs. The far source leaves
// of a chunk of the strong list are staged as one stream (a block scan of
// their counts places each source), 4T sources per pass across leaf
// boundaries, so that the pair loop mostly runs full runs and the barriers
// and staging are shared by several leaves; the near leaves form a second
// stream, 2T per pass. Per target the sources are summed in plain float over
// runs of 64 (full runs with a fixed trip count) and the runs compensated
// (Kahan).
template <typename OutT, int T>
__device__ __forceinline__ void p2p_f32_body(int B, int64_t n, const float *__restrict__ hl,
                                             const float *__restrict__ qf, const int32_t *__restrict__ begin,
                                             const int32_t *__restrict__ count, const float4 *__restrict__ geo,
                                             const int32_t *__restrict__ ssrc, const int4 unit, const int part,
                                             const int32_t *__restrict__ perm, const float *__restrict__ far_phi,
                                             const float *__restrict__ far_E, double4 *__restrict__ partial,
                                             OutT *__restrict__ pot, OutT *__restrict__ field) {
    constexpr int kP2PThreads = T, kFarCap = 4 * T, kNearCap = 2 * T;
    __shared__ float4 sA[kFarCap / 2], sB[kFarCap / 2];    // hi parts and charges, per source pair
    __shared__ float4 sC[kNearCap / 2], sD[kNearCap / 2];  // lo parts (near leaves)
    __shared__ float4 dh[kLeafChunk];   // per source leaf: centre offset hi, near flag
    __shared__ float4 dl[kLeafChunk];   // centre offset lo
    __shared__ int2 rng[kLeafChunk];    // begin, count
    __shared__ int fpre[kLeafChunk + 1];  // far leaves' counts (near: 0), then their exclusive prefix
    __shared__ int npre[kLeafChunk + 1];  // the same for the near leaves
    __shared__ int wsum[T / 32];
    static_assert(T == kP2PTile || T == kP2PTileSmall, "one target per thread");
    static_assert(kRun <= kNearCap && kNearCap <= kFarCap, "a run fits in a staged pass");
    const int64_t off = ((int64_t)1 << B) - 1;
    const int t = unit.x;
    const int64_t gt = off + t;
    const int bt = begin[gt], nt = count[gt];
    const int e0 = unit.z, e1 = unit.w;  // this unit's segment of the strong list
    const float4 tc_h = geo[3 * t], tc_l = geo[3 * t + 1], tc_e = geo[3 * t + 2];
    const int tid = threadIdx.x;
    const int i = unit.y + tid;
    const bool active = i < nt;
    // a warp with no target of the unit stages sources and keeps the barriers
    // but skips the products (the warps past a small leaf's last target)
    const bool busy = __any_sync(0xffffffffu, active);  // warp-uniform
    float xh = 0.f, yh = 0.f, zh = 0.f, xl = 0.f, yl = 0.f, zl = 0.f;
    if (active) {
        xh = hl[bt + i], yh = hl[n + bt + i], zh = hl[2 * n + bt + i];
        xl = hl[3 * n + bt + i], yl = hl[4 * n + bt + i], zl = hl[5 * n + bt + i];
    }
    const float2 X = make_float2(xh, xh), Y = make_float2(yh, yh), Z = make_float2(zh, zh);
    const float2 XL = make_float2(xl, xl), YL = make_float2(yl, yl), ZL = make_float2(zl, zl);
    float sum[4], comp[4];
#pragma unroll
    for (int j = 0; j < 4; j++) sum[j] = comp[j] = 0.f;
    float *fA = (float *)sA, *fB = (float *)sB, *fC = (float *)sC, *fD = (float *)sD;
    // runs of 64 staged sources (m of them from pair slot 0) against this
    // thread's target, each run compensated into the sums
    auto far_runs = [&](int m) {
        for (int j0 = 0; j0 < (busy ? m : 0); j0 += kRun) {
            const int npair = (min(kRun, m - j0) + 1) >> 1;
            const int p0 = j0 >> 1;
            float2 a[4];
#pragma unroll
            for (int c = 0; c < 4; c++) a[c] = make_float2(0.f, 0.f);
            if (npair == kRun / 2) {
#pragma unroll 8
                for (int pp = 0; pp < kRun / 2; pp++) far_pair2(X, Y, Z, sA[p0 + pp], sB[p0 + pp], a);
            } else {
#pragma unroll 4
                for (int pp = 0; pp < npair; pp++) far_pair2(X, Y, Z, sA[p0 + pp], sB[p0 + pp], a);
            }
#pragma unroll
            for (int c = 0; c < 4; c++) kahan(sum[c], comp[c], a[c].x + a[c].y);
        }
    };
    for (int cb = e0; cb < e1; cb += kLeafChunk) {
        const int clen = min(kLeafChunk, e1 - cb);
        __syncthreads();
        for (int k = tid; k < clen; k += kP2PThreads) {
            const int s = ssrc[cb + k];
            const float4 sh = geo[3 * s], sl = geo[3 * s + 1], se = geo[3 * s + 2];
            float e_x, e_y, e_z;
            const float dxh = two_sum(sh.x, -tc_h.x, e_x);
            const float dyh = two_sum(sh.y, -tc_h.y, e_y);
            const float dzh = two_sum(sh.z, -tc_h.z, e_z);
            const float gx = fmaxf(0.f, fabsf(dxh) - (tc_e.x + se.x));
            const float gy = fmaxf(0.f, fabsf(dyh) - (tc_e.y + se.y));
            const float gz = fmaxf(0.f, fabsf(dzh) - (tc_e.z + se.z));
            const float lim = kFarGap * (tc_h.w + sh.w);
            const bool far = gx * gx + gy * gy + gz * gz >= lim * lim && lim > 0.f;
            const int ns = count[off + s];
            dh[k] = make_float4(dxh, dyh, dzh, far ? 1.f : 0.f);
            dl[k] = make_float4(e_x + (sl.x - tc_l.x), e_y + (sl.y - tc_l.y), e_z + (sl.z - tc_l.z), 0.f);
            rng[k] = make_int2(begin[off + s], ns);
            fpre[k] = far ? ns : 0;
            npre[k] = far ? 0 : ns;
        }
        __syncthreads();
        block_excl_scan<T>(fpre, clen, wsum);
        block_excl_scan<T>(npre, clen, wsum);
        // far leaves: their sources as one stream, far source f of the chunk
        // in leaf kc with fpre[kc] <= f < fpre[kc + 1] (each thread's cursor
        // only moves forward)
        const int nfar = fpre[clen];
        int kc = 0;
        for (int base = 0; base < nfar; base += kFarCap) {
            __syncthreads();
#pragma unroll
            for (int r = 0; r < kFarCap / kP2PThreads; r++) {
                const int slot = r * kP2PThreads + tid, f = base + slot;
                float sx = kPadFar, sy = kPadFar, sz = kPadFar, q = 0.f;
                if (f < nfar) {
                    while (fpre[kc + 1] <= f) kc++;
                    const int bs = rng[kc].x + (f - fpre[kc]);
                    const float4 d = dh[kc], dlo = dl[kc];
                    sx = (hl[bs] + d.x) + (hl[3 * n + bs] + dlo.x);
                    sy = (hl[n + bs] + d.y) + (hl[4 * n + bs] + dlo.y);
                    sz = (hl[2 * n + bs] + d.z) + (hl[5 * n + bs] + dlo.z);
                    q = qf[bs];
                }
                const int sq = (slot >> 1) * 4 + (slot & 1);
                fA[sq] = -sx;
                fA[sq + 2] = -sy;
                fB[sq] = -sz;
                fB[sq + 2] = q;
            }
            __syncthreads();
            far_runs(min(kFarCap, nfar - base));
        }
        // near leaves: the second stream, with split hi/lo offsets
        const int nnear = npre[clen];
        kc = 0;
        for (int base = 0; base < nnear; base += kNearCap) {
            __syncthreads();
#pragma unroll
            for (int r = 0; r < kNearCap / kP2PThreads; r++) {
                const int slot = r * kP2PThreads + tid, f = base + slot;
                float sx = kPadFar, sy = kPadFar, sz = kPadFar, q = 0.f, ux = 0.f, uy = 0.f, uz = 0.f;
                if (f < nnear) {
                    while (npre[kc + 1] <= f) kc++;
                    const int bs = rng[kc].x + (f - npre[kc]);
                    const float4 d = dh[kc], dlo = dl[kc];
                    float ex, ey, ez;
                    sx = two_sum(hl[bs], d.x, ex);
                    sy = two_sum(hl[n + bs], d.y, ey);
                    sz = two_sum(hl[2 * n + bs], d.z, ez);
                    ux = ex + (hl[3 * n + bs] + dlo.x);
                    uy = ey + (hl[4 * n + bs] + dlo.y);
                    uz = ez + (hl[5 * n + bs] + dlo.z);
                    q = qf[bs];
                }
                const int sq = (slot >> 1) * 4 + (slot & 1);
                fA[sq] = -sx;
                fA[sq + 2] = -sy;
                fB[sq] = -sz;
                fB[sq + 2] = q;
                fC[sq] = -ux;
                fC[sq + 2] = -uy;
                fD[sq] = -uz;
            }
            __syncthreads();
            const int m = min(kNearCap, nnear - base);
            for (int j0 = 0; j0 < (busy ? m : 0); j0 += kRun) {
                const int npair = (min(kRun, m - j0) + 1) >> 1;
                const int p0 = j0 >> 1;
                float2 a[4];
#pragma unroll
                for (int c = 0; c < 4; c++) a[c] = make_float2(0.f, 0.f);
                if (npair == kRun / 2) {
#pragma unroll 8
                    for (int pp = 0; pp < kRun / 2; pp++)
                        near_pair2(X, Y, Z, XL, YL, ZL, sA[p0 + pp], sB[p0 + pp], sC[p0 + pp], sD[p0 + pp], a);
                } else {
#pragma unroll 4
                    for (int pp = 0; pp < npair; pp++)
                        near_pair2(X, Y, Z, XL, YL, ZL, sA[p0 + pp], sB[p0 + pp], sC[p0 + pp], sD[p0 + pp], a);
                }
#pragma unroll
                for (int c = 0; c < 4; c++) kahan(sum[c], comp[c], a[c].x + a[c].y);
            }
        }
    }
    if (active && part >= 0) {  // one segment of a split leaf: its partial sums
        partial[part + i] = make_double4((double)sum[0] - (double)comp[0], (double)sum[1] - (double)comp[1],
                                         (double)sum[2] - (double)comp[2], (double)sum[3] - (double)comp[3]);
    } else if (active) {
        const int64_t a = bt + i;
        const int64_t o = perm[a];
        pot[o] = (OutT)((double)far_phi[a] + ((double)sum[0] - (double)comp[0]));
        if (field) {
            field[3 * o] = (OutT)((double)far_E[a] + ((double)sum[1] - (double)comp[1]));
            field[3 * o + 1] = (OutT)((double)far_E[n + a] + ((double)sum[2] - (double)comp[2]));
            field[3 * o + 2] = (OutT)((double)far_E[2 * n + a] + ((double)sum[3] - (double)comp[3]));
        }
    }
}

// resident blocks asked of the register allocator (0: no constraint). The
// batched kernel holds the system's pointers in registers; unconstrained it
// takes 126 registers. At 64 registers for 128-target tiles (8 blocks) and 80
// for 64-target tiles (12 blocks) the 512-system batch ran in 319.0 ms, against
// 324.8 ms at 80 registers for both (328 ms at 72). The single-plan kernel runs
// best unconstrained (64 registers for 128-target tiles, 64 for 64: with 72 the
// 8M-point near field took 55.4 instead of 53.3 ms).
template <int T>
constexpr int p2p_min_blocks(bool batched) { return batched ? (T == kP2PTile ? 8 : 12) : 0; }

template <typename OutT, int T>
__global__ void __launch_bounds__(T, p2p_min_blocks<T>(false))
k_p2p_f32(int B, int64_t n, const float *__restrict__ hl, const float *__restrict__ qf,
          const int32_t *__restrict__ begin, const int32_t *__restrict__ count,
          const float4 *__restrict__ geo, const int32_t *__restrict__ ssrc, const int4 *__restrict__ units,
          const int32_t *__restrict__ upart, const int32_t *__restrict__ nunits,
          const int32_t *__restrict__ perm, const float *__restrict__ far_phi,
          const float *__restrict__ far_E, double4 *__restrict__ partial, OutT *__restrict__ pot,
          OutT *__restrict__ field) {
    if ((int)blockIdx.x >= *nunits) return;  // launched for an upper bound on the units
    p2p_f32_body<OutT, T>(B, n, hl, qf, begin, count, geo, ssrc, units[blockIdx.x], upart[blockIdx.x], perm,
                          far_phi, far_E, partial, pot, field);
}

// batched: the work units of every system in one list, heaviest first, each
// with its system
template <typename OutT, int T>
__global__ void __launch_bounds__(T, p2p_min_blocks<T>(true))
k_b_p2p_f32(const BatchSys *__restrict__ S, const int4 *__restrict__ units, const int32_t *__restrict__ usys,
            const int32_t *__restrict__ upart) {
    const BatchSys &y = S[usys[blockIdx.x]];
    p2p_f32_body<OutT, T>(y.B, y.n, y.hl, y.qf, y.begin, y.count, y.lgeo, y.ssrc, units[blockIdx.x],
                          upart[blockIdx.x], y.perm, y.far_phi, y.far_E, y.partial, (OutT *)y.pot, (OutT *)y.field);
}

}  // namespace

cudaError_t mixed_setup(Plan &P) {
    const int64_t n = P.n;
    P.hl = (float *)palloc(P, (size_t)n * 6 * 4);
    P.qf = (float *)palloc(P, (size_t)n * 4);
    P.far_phi_f = (float *)palloc(P, (size_t)n * 4);
    P.far_E_f = (float *)palloc(P, (size_t)n * 12);
    P.lgeo = (float4 *)palloc(P, (size_t)P.nleaf * 3 * sizeof(float4));
    if (!P.hl || !P.qf || !P.far_phi_f || !P.far_E_f || !P.lgeo) return cudaErrorMemoryAllocation;
    FMM_LAUNCH(k_leaf_offsets, (unsigned)P.nleaf, 128, 0, P.stream, P.B, n, P.x, P.y, P.z, P.begin,
               P.count, P.centre, P.hl);
    // half extents of the box that holds the leaf's points: its cell, or with
    // tight geometry the points' own bounding box
    FMM_LAUNCH(k_leaf_geo, (unsigned)((P.nleaf + 127) / 128), 128, 0, P.stream, P.B, P.tight ? P.tlo : P.lo,
               P.tight ? P.thi : P.hi, P.centre, P.radius, P.lgeo);
    return cudaGetLastError();
}

cudaError_t mixed_p2m(Plan &P, const void *charges, int dtype) {
    const int64_t n = P.n;
    const int gq = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
    if (dtype == FMM_F64)
        FMM_LAUNCH(k_gather_qf<double>, gq, 256, 0, P.stream, (const double *)charges, P.perm, P.qf, n);
    else
        FMM_LAUNCH(k_gather_qf<float>, gq, 256, 0, P.stream, (const float *)charges, P.perm, P.qf, n);
    FMM_LAUNCH(k_p2m_f32, (unsigned)P.nleaf, 32, sizeof(float2) * P.nc * 2,
               P.stream, P.B, P.p, n, P.hl, P.qf, P.begin, P.count, P.radius, P.M);
    return cudaGetLastError();
}

cudaError_t mixed_l2p(Plan &P) {
    FMM_LAUNCH(k_l2p_f32, (unsigned)P.nleaf, kThreads, sizeof(float2) * P.nc, P.stream, P.B, P.p,
               P.n, P.hl, P.begin, P.count, P.radius, P.L, P.far_phi_f, P.far_E_f);
    return cudaGetLastError();
}

template <int T>
static void launch_p2p_f32(Plan &P, void *pot, void *field, int dtype) {
    if (dtype == FMM_F64)
        FMM_LAUNCH((k_p2p_f32<double, T>), (unsigned)P.p2p_nunits, T, 0, P.stream, P.B, P.n, P.hl, P.qf, P.begin,
                   P.count, P.lgeo, P.ssrc[P.B], P.p2p_units, P.p2p_upart, P.p2p_nunits_dev, P.perm, P.far_phi_f,
                   P.far_E_f, P.p2p_partial, (double *)pot, (double *)field);
    else
        FMM_LAUNCH((k_p2p_f32<float, T>), (unsigned)P.p2p_nunits, T, 0, P.stream, P.B, P.n, P.hl, P.qf, P.begin,
                   P.count, P.lgeo, P.ssrc[P.B], P.p2p_units, P.p2p_upart, P.p2p_nunits_dev, P.perm, P.far_phi_f,
                   P.far_E_f, P.p2p_partial, (float *)pot, (float *)field);
}

cudaError_t mixed_p2p(Plan &P, void *pot, void *field, int dtype) {
    if (P.p2p_tile == kP2PTileSmall)
        launch_p2p_f32<kP2PTileSmall>(P, pot, field, dtype);
    else
        launch_p2p_f32<kP2PTile>(P, pot, field, dtype);
    return p2p_combine(P, pot, field, dtype);
}

// ---- batched stages
// (pmax: the largest order of the batch, for the shared-memory size)
cudaError_t batch_p2m(const BatchSys *S, const int32_t *off, int nsys, int64_t blocks, int pmax, cudaStream_t st) {
    if (blocks == 0) return cudaGetLastError();
    FMM_LAUNCH(k_b_p2m_f32, (unsigned)blocks, 32, sizeof(float2) * ncoef(pmax) * 2, st, S, off, nsys);
    return cudaGetLastError();
}

cudaError_t batch_l2p(const BatchSys *S, const int32_t *off, int nsys, int64_t blocks, int pmax, cudaStream_t st) {
    if (blocks == 0) return cudaGetLastError();
    FMM_LAUNCH(k_b_l2p_f32, (unsigned)blocks, kThreads, sizeof(float2) * ncoef(pmax), st, S, off, nsys);
    return cudaGetLastError();
}

cudaError_t batch_p2p(const BatchSys *S, const int4 *units, const int32_t *usys, const int32_t *upart, int64_t n,
                      int tile, int dtype, cudaStream_t st) {
    if (n == 0) return cudaGetLastError();
    if (tile == kP2PTileSmall) {
        if (dtype == FMM_F64)
            FMM_LAUNCH((k_b_p2p_f32<double, kP2PTileSmall>), (unsigned)n, kP2PTileSmall, 0, st, S, units, usys, upart);
        else
            FMM_LAUNCH((k_b_p2p_f32<float, kP2PTileSmall>), (unsigned)n, kP2PTileSmall, 0, st, S, units, usys, upart);
    } else {
        if (dtype == FMM_F64)
            FMM_LAUNCH((k_b_p2p_f32<double, kP2PTile>), (unsigned)n, kP2PTile, 0, st, S, units, usys, upart);
        else
            FMM_LAUNCH((k_b_p2p_f32<float, kP2PTile>), (unsigned)n, kP2PTile, 0, st, S, units, usys, upart);
    }
    return cudaGetLastError();
}

}  // namespace fmm
