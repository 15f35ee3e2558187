// M2L on the tensor cores: tcgen05.mma kind::tf32 with FP32 accumulation in
// tensor memory, three products per contraction for single-precision
// accuracy.
//
// The rotational M2L (Sec. 2.1.3) of one weak pair is a chain of products of
// fixed small matrices with per-pair vectors: per degree n the two folds with
// d^n(pi/2) of the forward y-rotation, per order l the axial translation, per
// degree the two folds of the inverse rotation (65 contractions at p = 12).
// Stacking 128 pairs as the rows of A turns each of them into one
// [128 x K] x [K x 16] tensor-core product (K = n+1 or p+1-l rounded up to
// 8); the per-pair diagonal factors between the products (z-rotations, box
// ratio powers, the i^m phases) stay with the thread that owns the pair.
// The scaled forms are those of the single-precision SIMT kernel: the source
// multipole is read as M_n / r_s^n and the result accumulated as r_t^k L_k.
//
// Numerics: every operand is split into tf32 hi + lo parts (round to
// nearest) and a contraction is A_hi B_hi + A_hi B_lo + A_lo B_hi, summed in
// FP32 by the tensor core: ~3e-7 relative per product.
//
// Layout (one CTA of 256 threads per SM, persistent over tiles of pairs):
//  - two teams of 128 threads; thread i of a team owns pair i of the team's
//    tile, row i of A and lane i of the team's accumulators;
//  - tensor memory, 256 columns per team: the pair's rotated coefficients
//    V (real parts at column tri(n,m), imaginary at 96 + tri(n,m)), A_hi
//    (Re [192,208), Im [208,224)) and the results (Re [224,240), Im
//    [240,256));
//  - shared memory: the fixed B matrices (hi and lo, K-major, no swizzle:
//    core matrices of 8 rows x 16 bytes, LBO 128 B along K, SBO 32 Kp B
//    along the rows), A_lo of each team (same layout, 128 x 16, Re and
//    Im), and a per-warp transpose buffer for the reduction of contributions
//    to one target;
//  - one thread per team issues the team's MMAs and commits them to the
//    team's mbarrier; every wait has an iteration limit, after which the
//    team sets the plan's error word and stops.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "fmm_internal.cuh"
#include "m2l_common.cuh"

namespace fmm {

namespace {

constexpr int kTeam = 128;
constexpr int kTcThreads = 2 * kTeam;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kTeamCols = 256;
constexpr int kTcPMax = 12;          // 2 (p+1)(p+2)/2 <= 192 columns of V
constexpr uint32_t kVIm = 96, kAHi = 192, kDst = 224;
constexpr int kRedStride = 36;        // floats per row of the reduction buffer
constexpr uint32_t kSpinLimit = 1u << 24;

__host__ __device__ constexpr int kpad(int len) { return (len + 7) & ~7; }
// one 16 x Kp matrix, bytes
__host__ __device__ constexpr int mat_bytes(int len) { return 16 * kpad(len) * 4; }
// byte offset of (row o, column k) in a K-major 16 x Kp matrix
__host__ __device__ constexpr int elem_off(int o, int k, int kp) {
    return (o & 7) * 16 + (o >> 3) * (kp * 32) + (k & 3) * 4 + (k >> 2) * 128;
}
// table layout for order p: per degree n eight matrices (fold / fold^T x
// Re / Im x hi / lo), then per order l two (axial hi / lo)
__host__ __device__ constexpr int deg_off(int n) {
    int o = 0;
    for (int j = 0; j < n; j++) o += 8 * mat_bytes(j + 1);
    return o;
}
__host__ __device__ constexpr int ax_off(int p, int l) {
    int o = deg_off(p + 1);
    for (int j = 0; j < l; j++) o += 2 * mat_bytes(p + 1 - j);
    return o;
}
__host__ __device__ constexpr int tab_bytes(int p) { return ax_off(p, p + 1); }
constexpr int kALoBytes = kTeam * 16 * 4;  // one 128 x 16 K-major matrix
constexpr int kRedBytes = 8 * 32 * kRedStride * 4;

__host__ __device__ constexpr int smem_bytes(int p) { return tab_bytes(p) + 4 * kALoBytes + kRedBytes; }

// ---- PTX wrappers ---------------------------------------------------------
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// kind::tf32, D f32, A and B tf32 K-major, M = 128, N = 16
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void st16(uint32_t taddr, const float (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]),
        "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]));
}

__device__ __forceinline__ void st1(uint32_t taddr, float v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "f"(v));
}

__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float ld1(uint32_t taddr) {
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    return __uint_as_float(r);
}

__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void team_sync(int team) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + team), "r"(kTeam) : "memory");
}

// barrier of the team's 128 threads that also ANDs a flag over them, so that
// every thread of the team takes the same branch afterwards
__device__ __forceinline__ bool team_all(int team, bool v) {
    uint32_t r;
    asm volatile(
        "{\n.reg .pred q, r;\nsetp.ne.u32 q, %1, 0;\nbar.red.and.pred r, %2, %3, q;\nselp.u32 %0, 1, 0, r;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(1 + team), "r"(kTeam)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < kSpinLimit && !done; it++) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
    }
    return done != 0;
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 ipowf(int m, float2 v) {  // i^m v
    switch (m & 3) {
        case 0: return v;
        case 1: return make_float2(-v.y, v.x);
        case 2: return make_float2(-v.x, -v.y);
        default: return make_float2(v.y, -v.x);
    }
}

__constant__ float c_tcF[(kTcPMax + 1) * (kTcPMax + 2) / 2];  // F_nm

// Per-team state.
struct Team {
    uint32_t tcol;      // team's first tensor-memory column (lane field 0)
    uint32_t lanes;     // this warp's lane quarter, in the address's lane field
    uint32_t bar;       // the team's mbarrier (shared address)
    uint32_t phase;
    uint32_t tab;       // shared address of the B tables
    float *alo;         // this team's A_lo (Re at +0, Im at +kALoBytes)
    int id;
    int row;
    bool leader;
    volatile int *abort;  // shared flag: a wait ran out
};

// One contraction for the team: (re, im) rows of A in, (re, im) rows of
// D = A B^T out, with B given by the shared addresses of its hi and lo parts
// (bre: Re, bim: Im; each 16 x kp) and kp in {8, 16}.
__device__ __forceinline__ bool contract(Team &T, float (&re)[16], float (&im)[16], uint32_t bre_hi,
                                         uint32_t bre_lo, uint32_t bim_hi, uint32_t bim_lo, int kp,
                                         int *err) {
    float h[16];
    {
        float lo[16];
#pragma unroll
        for (int j = 0; j < 16; j++) {
            h[j] = tf32_rn(re[j]);
            lo[j] = tf32_rn(re[j] - h[j]);
        }
        st16(T.tcol + T.lanes + kAHi, h);
        char *base = (char *)T.alo + (T.row & 7) * 16 + (T.row >> 3) * 512;
#pragma unroll
        for (int q = 0; q < 4; q++)
            *(float4 *)(base + q * 128) = make_float4(lo[4 * q], lo[4 * q + 1], lo[4 * q + 2], lo[4 * q + 3]);
#pragma unroll
        for (int j = 0; j < 16; j++) {
            h[j] = tf32_rn(im[j]);
            lo[j] = tf32_rn(im[j] - h[j]);
        }
        st16(T.tcol + T.lanes + kAHi + 16, h);
        base += kALoBytes;
#pragma unroll
        for (int q = 0; q < 4; q++)
            *(float4 *)(base + q * 128) = make_float4(lo[4 * q], lo[4 * q + 1], lo[4 * q + 2], lo[4 * q + 3]);
    }
    wait_st();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    team_sync(T.id);
    const bool go = !*T.abort;
    if (T.leader && go) {
        fence_after();
        const uint32_t sbo = (uint32_t)kp * 32;
        const uint32_t alo = su32(T.alo);
        for (int kb = 0; kb < kp / 8; kb++) {
            const uint32_t ko = 256u * kb;
            mma_ts(T.tcol + kDst, T.tcol + kAHi + 8 * kb, sdesc(bre_hi + ko, sbo), kb > 0);
            mma_ts(T.tcol + kDst, T.tcol + kAHi + 8 * kb, sdesc(bre_lo + ko, sbo), 1);
            mma_ss(T.tcol + kDst, sdesc(alo + ko, 512), sdesc(bre_hi + ko, sbo), 1);
            mma_ts(T.tcol + kDst + 16, T.tcol + kAHi + 16 + 8 * kb, sdesc(bim_hi + ko, sbo), kb > 0);
            mma_ts(T.tcol + kDst + 16, T.tcol + kAHi + 16 + 8 * kb, sdesc(bim_lo + ko, sbo), 1);
            mma_ss(T.tcol + kDst + 16, sdesc(alo + kALoBytes + ko, 512), sdesc(bim_hi + ko, sbo), 1);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(T.bar)
                     : "memory");
    }
    bool ok = go && mbar_wait(T.bar, T.phase);
    if (go) T.phase ^= 1u;
    ok = team_all(T.id, ok);
    if (!ok) {
        if (T.leader) {
            *T.abort = 1;
            atomicOr(err, 16);
        }
        return false;
    }
    fence_after();
    ld16(T.tcol + T.lanes + kDst, re);
    ld16(T.tcol + T.lanes + kDst + 16, im);
    wait_ld();
    // the loaded registers are valid only after the wait: tie their uses to it
#pragma unroll
    for (int j = 0; j < 16; j++) asm volatile("" : "+f"(re[j]), "+f"(im[j]));
    return true;
}

// Sum over the warp's pairs of one degree's contributions (2 (n+1) values
// per lane, Re in val[0..n], Im in val[16..16+n]) into Lh of their target.
// A warp whose valid lanes share one target transposes through shared
// memory; otherwise the segmented shuffle sum of runs of equal target.
__device__ __forceinline__ void reduce_out(int n, const float (&vr)[16], const float (&vi)[16], int64_t gt,
                                           double2 *__restrict__ Lh, int nc, float *red,
                                           const bool (&same)[5], bool head) {
    const int lane = threadIdx.x & 31;
    const int t32 = gt >= 0 ? (int)gt : -1;
    const int tmax = __reduce_max_sync(0xffffffffu, t32);
    const bool uniform = __all_sync(0xffffffffu, t32 == tmax || t32 < 0);
    const int c0 = n * (n + 1) / 2;
    if (uniform) {
        if (tmax < 0) return;
        float *row = red + lane * kRedStride;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            *(float4 *)(row + 4 * q) = make_float4(vr[4 * q], vr[4 * q + 1], vr[4 * q + 2], vr[4 * q + 3]);
            *(float4 *)(row + 16 + 4 * q) = make_float4(vi[4 * q], vi[4 * q + 1], vi[4 * q + 2], vi[4 * q + 3]);
        }
        __syncwarp();
        const int col = lane < n + 1 ? lane : (lane < 2 * (n + 1) ? 16 + lane - (n + 1) : -1);
        if (col >= 0) {
            float s = 0.f;
#pragma unroll 8
            for (int i = 0; i < 32; i++) s += red[i * kRedStride + col];
            double *dst = (double *)&Lh[(int64_t)tmax * nc + c0 + (col & 15)];
            atomicAdd(dst + (col >= 16 ? 1 : 0), (double)s);
        }
        __syncwarp();
    } else {
#pragma unroll
        for (int l = 0; l < 16; l++) {
            if (l > n) break;
            const float rx = seg_sum(vr[l], same), ry = seg_sum(vi[l], same);
            if (head) {
                atomicAdd(&Lh[gt * nc + c0 + l].x, (double)rx);
                atomicAdd(&Lh[gt * nc + c0 + l].y, (double)ry);
            }
        }
    }
}

__global__ void __launch_bounds__(kTcThreads, 1)
k_m2l_tc(PairTable PT, int p, int64_t ntiles, const float4 *__restrict__ cf, const float2 *__restrict__ Mf,
         double2 *__restrict__ Lh,
         const uint4 *__restrict__ gtab, int *err) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ int s_abort[2];
    const int tid = threadIdx.x, team = tid / kTeam, row = tid % kTeam, warp = tid >> 5;
    const int nc = ncoef(p);
    const int tb = tab_bytes(p);
    // fixed matrices into shared memory
    for (int i = tid; i < tb / 16; i += kTcThreads) ((uint4 *)tc_smem)[i] = gtab[i];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&s_bar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&s_bar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_abort[0] = s_abort[1] = 0;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();

    Team T;
    T.tcol = s_tmem + kTeamCols * team;
    T.lanes = (uint32_t)(32 * (warp & 3)) << 16;
    T.bar = su32(&s_bar[team]);
    T.phase = 0;
    T.tab = su32(tc_smem);
    T.alo = (float *)(tc_smem + tb + 2 * kALoBytes * team);
    T.id = team;
    T.row = row;
    T.leader = row == 0;
    T.abort = &s_abort[team];
    float *red = (float *)(tc_smem + tb + 4 * kALoBytes) + warp * 32 * kRedStride;
    const uint32_t vre = T.tcol + T.lanes, vim = T.tcol + T.lanes + kVIm;
    const int64_t tot = PT.off[PT.lmax + 1];

    for (int64_t tile = (int64_t)blockIdx.x * 2 + team; tile < ntiles; tile += (int64_t)gridDim.x * 2) {
        if (*T.abort) break;
        const int64_t g = tile * kTeam + row;
        const bool valid = g < tot;
        int64_t gt = -1, gs = 0;
        float dx = 1.f, dy = 0.f, dz = 0.f, rs = 1.f, rt = 1.f;
        if (valid) {
            pair_of(PT, g, gt, gs);
            // the offset from the split float centres, as the CUDA-core kernel forms it
            const float4 th = cf[2 * gt], tl = cf[2 * gt + 1], sh = cf[2 * gs], sl = cf[2 * gs + 1];
            dx = offset_f(th.x, sh.x, tl.x, sl.x);
            dy = offset_f(th.y, sh.y, tl.y, sl.y);
            dz = offset_f(th.z, sh.z, tl.z, sl.z);
            rs = sh.w > 0.f ? sh.w : 1.f;
            rt = th.w > 0.f ? th.w : 1.f;
        }
        bool same[5], head;
        seg_setup(gt, same, head);
        const float rxy2 = fmaf(dx, dx, dy * dy);
        const float rxy = sqrtf(rxy2), rinv = rsqrtf(fmaf(dz, dz, rxy2));
        const float rxinv = rxy > 0.f ? 1.f / rxy : 0.f;
        const float2 ea = rxy > 0.f ? make_float2(dx * rxinv, dy * rxinv) : make_float2(1.f, 0.f);
        const float2 ebv = make_float2(dz * rinv, rxy * rinv);
        const float2 eai = make_float2(ea.y, -ea.x);
        const float qs = rs * rinv, qt = rt * rinv;
        const float2 *Ms = Mf + (valid ? gs : 0) * mf_stride(p);
        bool ok = true;

        // 1-2. forward rotation, degree by degree: V_n = i^m fold^T(e^{ikb} fold(F e^{ima} M_n))
        for (int n = 0; n <= p && ok; n++) {
            float re[16], im[16];
            const int c0 = n * (n + 1) / 2;
            float2 ph = make_float2(1.f, 0.f);
#pragma unroll
            for (int m = 0; m < 16; m++) {
                re[m] = 0.f;
                im[m] = 0.f;
                if (m <= n) {
                    const float2 mv = valid ? Ms[c0 + m] : make_float2(0.f, 0.f);
                    const float s = c_tcF[c0 + m] * (m ? 2.f : 1.f);
                    const float2 t = cmulf(mv, ph);
                    re[m] = t.x * s;
                    im[m] = t.y * s;
                    ph = cmulf(ph, eai);
                }
            }
            const uint32_t dn = T.tab + deg_off(n), mb = mat_bytes(n + 1);
            const int kp = kpad(n + 1);
            ok = contract(T, re, im, dn, dn + mb, dn + 2 * mb, dn + 3 * mb, kp, err);
            if (!ok) break;
            float2 pb = make_float2(1.f, 0.f);
#pragma unroll
            for (int k = 0; k < 16; k++) {
                if (k <= n) {
                    const float2 t = cmulf(make_float2(re[k], im[k]), pb);
                    const float f = k ? 2.f : 1.f;
                    re[k] = t.x * f;
                    im[k] = t.y * f;
                    pb = cmulf(pb, ebv);
                } else {
                    re[k] = 0.f;
                    im[k] = 0.f;
                }
            }
            ok = contract(T, re, im, dn + 4 * mb, dn + 5 * mb, dn + 6 * mb, dn + 7 * mb, kp, err);
            if (!ok) break;
#pragma unroll
            for (int m = 0; m < 16; m++) {
                const float2 v = ipowf(m, make_float2(re[m], im[m]));
                re[m] = v.x;
                im[m] = v.y;
            }
            // 16 columns from tri(n, 0): the ones past degree n belong to
            // higher degrees, which are written later
            st16(vre + c0, re);
            st16(vim + c0, im);
            wait_st();
        }
        // 3. translation along z, order by order (in place in V)
        for (int l = 0; l <= p && ok; l++) {
            float re[16], im[16];
            float sp = 1.f;
            for (int j = 0; j < l; j++) sp *= qs;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int n = l + j;
                if (n <= p) {
                    const int c = n * (n + 1) / 2 + l;
                    re[j] = ld1(vre + c);
                    im[j] = ld1(vim + c);
                } else {
                    re[j] = 0.f;
                    im[j] = 0.f;
                }
            }
            wait_ld();
#pragma unroll
            for (int j = 0; j < 16; j++) asm volatile("" : "+f"(re[j]), "+f"(im[j]));
#pragma unroll
            for (int j = 0; j < 16; j++) {
                if (l + j <= p) {
                    re[j] = re[j] * sp;
                    im[j] = -im[j] * sp;
                    sp *= qs;
                }
            }
            const uint32_t ab = T.tab + ax_off(p, l), mb = mat_bytes(p + 1 - l);
            ok = contract(T, re, im, ab, ab + mb, ab, ab + mb, kpad(p + 1 - l), err);
            if (!ok) break;
            float tp = rinv;
            for (int j = 0; j < l; j++) tp *= qt;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int k = l + j;
                if (k <= p) {
                    const int c = k * (k + 1) / 2 + l;
                    st1(vre + c, re[j] * tp);
                    st1(vim + c, im[j] * tp);
                    tp *= qt;
                }
            }
            wait_st();
        }
        // 4-5. inverse rotation, degree by degree, and the reduction into Lh
        for (int n = 0; n <= p && ok; n++) {
            float re[16], im[16];
            const int c0 = n * (n + 1) / 2;
            ld16(vre + c0, re);
            ld16(vim + c0, im);
            wait_ld();
#pragma unroll
            for (int j = 0; j < 16; j++) asm volatile("" : "+f"(re[j]), "+f"(im[j]));
#pragma unroll
            for (int m = 0; m < 16; m++) {
                if (m <= n) {
                    const float2 t = ipowf(m, make_float2(re[m], im[m]));
                    const float f = m ? 2.f : 1.f;
                    re[m] = t.x * f;
                    im[m] = t.y * f;
                } else {
                    re[m] = 0.f;
                    im[m] = 0.f;
                }
            }
            const uint32_t dn = T.tab + deg_off(n), mb = mat_bytes(n + 1);
            const int kp = kpad(n + 1);
            ok = contract(T, re, im, dn, dn + mb, dn + 2 * mb, dn + 3 * mb, kp, err);
            if (!ok) break;
            float2 pb = make_float2(1.f, 0.f);
#pragma unroll
            for (int k = 0; k < 16; k++) {
                if (k <= n) {
                    const float2 t = cmulf(make_float2(re[k], im[k]), pb);
                    const float f = k ? 2.f : 1.f;
                    re[k] = t.x * f;
                    im[k] = t.y * f;
                    pb = cmulf(pb, ebv);
                } else {
                    re[k] = 0.f;
                    im[k] = 0.f;
                }
            }
            ok = contract(T, re, im, dn + 4 * mb, dn + 5 * mb, dn + 6 * mb, dn + 7 * mb, kp, err);
            if (!ok) break;
            float2 ph = make_float2(1.f, 0.f);
#pragma unroll
            for (int l = 0; l < 16; l++) {
                if (l <= n) {
                    const float2 t = cmulf(ipowf(4 - (l & 3), make_float2(re[l], im[l])), ph);
                    const float f = c_tcF[c0 + l];
                    re[l] = valid ? t.x * f : 0.f;
                    im[l] = valid ? t.y * f : 0.f;
                    ph = cmulf(ph, ea);
                } else {
                    re[l] = 0.f;
                    im[l] = 0.f;
                }
            }
            reduce_out(n, re, im, gt, Lh, nc, red, same, head);
        }
        if (!ok) break;
    }
    fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(kTmemCols));
}

// host: tf32 round to nearest (ties away), as cvt.rna
float tf32_host(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;
    u = (u + 0x1000u) & 0xffffe000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// The B image for order p: shared-memory byte layout, as floats.
std::vector<float> tc_tables(int p) {
    std::vector<float> img((size_t)tab_bytes(p) / 4, 0.f);
    auto put = [&](int base, int kp, int o, int k, long double v, bool lo) {
        const float hi = tf32_host((float)v);
        const float x = lo ? tf32_host((float)(v - (long double)hi)) : hi;
        img[(size_t)(base + elem_off(o, k, kp)) / 4] = x;
    };
    for (int n = 0; n <= p; n++) {
        const int kp = kpad(n + 1), mb = mat_bytes(n + 1);
        for (int stage = 0; stage < 2; stage++)
            for (int part = 0; part < 2; part++)
                for (int hl = 0; hl < 2; hl++) {
                    const int base = deg_off(n) + ((stage * 2 + part) * 2 + hl) * mb;
                    for (int o = 0; o <= n; o++)
                        for (int k = 0; k <= n; k++) {
                            if (((n + o + k) & 1) != part) continue;  // Re: even parity, Im: odd
                            // fold: out_o = sum_k D[o][k] v_k; fold^T: out_o = sum_k D[k][o] v_k
                            const long double d = stage == 0 ? wigner_half_pi(n, o, k) : wigner_half_pi(n, k, o);
                            put(base, kp, o, k, d, hl == 1);
                        }
                }
    }
    auto F = [](int n, int m) { return sqrtl(factl(n + m) * factl(n - m)); };
    for (int l = 0; l <= p; l++) {
        const int len = p + 1 - l, kp = kpad(len), mb = mat_bytes(len);
        for (int hl = 0; hl < 2; hl++) {
            const int base = ax_off(p, l) + hl * mb;
            for (int o = 0; o < len; o++)
                for (int k = 0; k < len; k++) {
                    const int kk = l + o, nn = l + k;
                    long double a = factl(nn + kk) / (F(nn, l) * F(kk, l));
                    if ((kk + l) & 1) a = -a;
                    put(base, kp, o, k, a, hl == 1);
                }
        }
    }
    return img;
}

struct TcTabCache {
    void *dev[64][kTcPMax + 1] = {};
    bool fready[64] = {};
};
TcTabCache g_tc;
std::atomic<int> g_tc_lock{0};

}  // namespace

bool m2l_tc_supported(int p) { return p >= 1 && p <= kTcPMax; }

// plan-time: tables on the device (once per device and order), the kernel's
// shared-memory attribute, and the CTA count
cudaError_t m2l_tc_setup(Plan &P) {
    if (!m2l_tc_supported(P.p)) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    while (g_tc_lock.exchange(1, std::memory_order_acquire)) {
    }
    if (!g_tc.fready[dev]) {
        std::vector<float> F;
        for (int n = 0; n <= kTcPMax; n++)
            for (int m = 0; m <= n; m++) F.push_back((float)sqrtl(factl(n + m) * factl(n - m)));
        e = cudaMemcpyToSymbol(c_tcF, F.data(), F.size() * 4);
        if (e == cudaSuccess) g_tc.fready[dev] = true;
    }
    if (e == cudaSuccess && !g_tc.dev[dev][P.p]) {
        const std::vector<float> img = tc_tables(P.p);
        void *d = nullptr;
        e = cudaMalloc(&d, img.size() * 4);
        if (e == cudaSuccess) e = cudaMemcpy(d, img.data(), img.size() * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            g_tc.dev[dev][P.p] = d;
        else if (d)
            cudaFree(d);
    }
    g_tc_lock.store(0, std::memory_order_release);
    if (e != cudaSuccess) return e;
    P.tc_tab = g_tc.dev[dev][P.p];
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    P.tc_ctas = sms;
    return allow_max_smem((const void *)k_m2l_tc, smem_bytes(P.p));
}

// the weak pairs of all levels through the tensor cores; accumulates the
// scaled locals into Lh (zeroed by the caller)
cudaError_t m2l_tc_launch(Plan &P) {
    const int64_t tot = total_weak(P);
    if (tot == 0) return cudaSuccess;
    const int64_t ntiles = (tot + kTeam - 1) / kTeam;
    const int grid = (int)std::min<int64_t>(P.tc_ctas, (ntiles + 1) / 2);
    FMM_LAUNCH(k_m2l_tc, grid, kTcThreads, smem_bytes(P.p), P.stream, pair_table(P), P.p, ntiles, P.box_cf, P.Mf,
               P.Lh, (const uint4 *)P.tc_tab, P.d_err + 1);
    return cudaGetLastError();
}

}  // namespace fmm
