// M2L in the rotational form the paper uses (Sec. 2.1.3: rotate the z-axis of
// the expansion onto the box-to-box vector, translate along it, rotate back;
// O(p^3) per weak pair instead of O(p^4)).
//
// With d = c_t - c_s = rho (sin b cos a, sin b sin a, cos b) and the
// normalisation F_nm = sqrt((n+|m|)! (n-|m|)!), a multipole M_n^m of the
// source becomes a local expansion L_k^l of the target by
//   1. u_m   = F_nm M_n^m e^{i m a}                    z-rotation (diagonal)
//   2. Mr_n  = d^n(b)^T u                              y-rotation, per degree
//   3. Lr_k^l = sum_n (-1)^(k+l) (n+k)!/(F_nl F_kl) rho^-(n+k+1) conj(Mr_n^l)
//                                                     translation along z
//   4. Lb_k  = d^k(b) Lr_k                             inverse y-rotation
//   5. L_k^l += F_kl e^{i l a} Lb_k^l                  inverse z-rotation
// and the y-rotation factors through the fixed matrix D = d^n(pi/2)
// (Pinchon & Hoggan):  d_{m'm}(b) = sum_k i^{m-m'} D_{km'} D_{km} e^{ikb}.
// Every vector has the real-source symmetry v_{-m} = (-1)^m conj(v_m), and
// D_{k,-m} = (-1)^{n+k} D_{km}, so a product with D folds onto m, k >= 0:
//   out_k = sum_{m = n+k mod 2} D_km Re v_m + i sum_{m != n+k mod 2} D_km Im v_m
// with v_m doubled for m > 0: (n+1)^2 real multiply-adds per degree.
//
// GPU mapping (double precision): GB300's FP64 pipe retires about two
// multiply-adds per clock per SM, so the kernel is organised to issue as few
// FP64 instructions as possible and lets everything else be cheap: one CTA
// per target box, one weak pair per thread, per-thread coefficient vectors
// in shared memory (column per thread, conflict-free), D and the axial
// coefficients in shared memory (every lane reads the same entry: broadcast),
// and a warp shuffle reduction of the contributions into a per-warp
// accumulator, so no atomics are needed.

#include <algorithm>
#include <cmath>
#include <atomic>
#include <mutex>
#include <vector>

#include "fmm_internal.cuh"
#include "m2l_common.cuh"

namespace fmm {

namespace {

__device__ __forceinline__ double2 mul_ipow(int m, double2 v) {  // i^m v
    switch (m & 3) {
        case 0: return v;
        case 1: return make_double2(-v.y, v.x);
        case 2: return make_double2(-v.x, -v.y);
        default: return make_double2(v.y, -v.x);
    }
}

// out_k (k = 0..n) = fold(D^n) applied to v (m = 0..n); transpose: use D_mk.
__device__ __forceinline__ void fold_apply(const double *__restrict__ D, int n, const double2 *v,
                                           double2 *out, int stride, bool transpose) {
    for (int k = 0; k <= n; k++) {
        double re = 0.0, im = 0.0;
        const int par = (n + k) & 1;
        for (int m = par; m <= n; m += 2)
            re = fma(transpose ? D[m * (n + 1) + k] : D[k * (n + 1) + m], v[m * stride].x, re);
        for (int m = 1 - par; m <= n; m += 2)
            im = fma(transpose ? D[m * (n + 1) + k] : D[k * (n + 1) + m], v[m * stride].y, im);
        out[k * stride] = make_double2(re, im);
    }
}

// With ext_M set, the sources are not boxes of the plan: pair g is (target
// box PT.tgt[PT.lmin][g] of level PT.lmin, source g with multipole ext_M[g]
// about ext_centre[g]) -- a split system's multipoles from another rank; the
// targets are then in no particular order, so each pair adds its own result.
__global__ void k_m2l_rot_f64(PairTable PT, int p, const double *__restrict__ centre,
                              const double2 *__restrict__ M, double2 *__restrict__ L,
                              const double *__restrict__ gtab, int ntab,
                              const double *__restrict__ ext_centre = nullptr,
                              const double2 *__restrict__ ext_M = nullptr) {
    extern __shared__ double2 sm2[];
    const int nc = ncoef(p), T = blockDim.x, tid = threadIdx.x;
    // shared layout: [V: nc*T][U: (p+1)*T][W: (p+1)*T][tables: ntab doubles]
    double2 *V = sm2;
    double2 *U = V + nc * T;
    double2 *W = U + (p + 1) * T;
    double *tab = (double *)(W + (p + 1) * T);
    for (int i = tid; i < ntab; i += T) tab[i] = gtab[i];
    __syncthreads();
    // tables: D (sum (n+1)^2), axial A (sum_l (p+1-l)^2), F_nm (nc)
    const double *Dt = tab;
    const int nD = (p + 1) * (p + 2) * (2 * p + 3) / 6;
    const double *At = Dt + nD;
    const double *Ft = At + nD;
    double2 *v = V + tid, *u = U + tid, *x = W + tid;

    const int64_t g = blockIdx.x * (int64_t)T + tid;
    const bool valid = g < PT.off[PT.lmax + 1];
    int64_t gt = -1, gs = 0;
    double dx = 1.0, dy = 0.0, dz = 0.0;
    const double *cs = ext_M ? ext_centre : centre;
    const double2 *Ms = ext_M ? ext_M : M;
    if (valid) {
        if (ext_M) {
            gt = ((int64_t)1 << PT.lmin) - 1 + PT.tgt[PT.lmin][g];
            gs = g;
        } else {
            pair_of(PT, g, gt, gs);
        }
        dx = centre[3 * gt] - cs[3 * gs];
        dy = centre[3 * gt + 1] - cs[3 * gs + 1];
        dz = centre[3 * gt + 2] - cs[3 * gs + 2];
    }
    bool same[5], head;
    seg_setup(gt, same, head);
    if (ext_M) {  // external pairs come in any order: no run sums, one atomic add per pair
#pragma unroll
        for (int j = 0; j < 5; j++) same[j] = false;
        head = valid;
    }
    const double rxy = sqrt(dx * dx + dy * dy);
    const double rho = sqrt(dx * dx + dy * dy + dz * dz);
    const double rinv = 1.0 / rho;
    const double2 ea = rxy > 0.0 ? make_double2(dx / rxy, dy / rxy) : make_double2(1.0, 0.0);
    const double2 eb_ = make_double2(dz * rinv, rxy * rinv);
    const double2 eai = make_double2(ea.y, -ea.x);  // -i e^{ia}

    // ---- forward rotation, degree by degree -> v = Mr (F-normalised)
    const double *Dn = Dt;
    for (int n = 0; n <= p; n++) {
        double2 ph = make_double2(1.0, 0.0);
        for (int m = 0; m <= n; m++) {
            const int c = tri(n, m);
            const double2 mv = valid ? Ms[gs * nc + c] : make_double2(0.0, 0.0);
            u[m * T] = cscale(cmul(mv, ph), Ft[c] * (m ? 2.0 : 1.0));
            ph = cmul(ph, eai);
        }
        fold_apply(Dn, n, u, x, T, false);
        double2 pb = make_double2(1.0, 0.0);
        for (int k = 0; k <= n; k++) {
            x[k * T] = cscale(cmul(x[k * T], pb), k ? 2.0 : 1.0);
            pb = cmul(pb, eb_);
        }
        fold_apply(Dn, n, x, u, T, true);
        for (int m = 0; m <= n; m++) v[tri(n, m) * T] = mul_ipow(m, u[m * T]);
        Dn += (n + 1) * (n + 1);
    }
    // ---- translation along z, order by order (in place)
    const double *Al = At;
    double rl = 1.0;  // rho^-l
    for (int l = 0; l <= p; l++) {
        const int len = p + 1 - l;
        double rp = rl;
        for (int n = l; n <= p; n++) {
            const double2 mr = v[tri(n, l) * T];
            u[(n - l) * T] = make_double2(mr.x * rp, -mr.y * rp);
            rp *= rinv;
        }
        double rk = rl * rinv;  // rho^-(k+1) at k = l
        for (int k = l; k <= p; k++) {
            double re = 0.0, im = 0.0;
            const double *a = Al + (k - l) * len;
            for (int j = 0; j < len; j++) {
                const double2 s = u[j * T];
                re = fma(a[j], s.x, re);
                im = fma(a[j], s.y, im);
            }
            v[tri(k, l) * T] = make_double2(re * rk, im * rk);
            rk *= rinv;
        }
        Al += len * len;
        rl *= rinv;
    }
    // ---- inverse rotation, degree by degree; segmented reduction per target
    Dn = Dt;
    for (int k = 0; k <= p; k++) {
        for (int m = 0; m <= k; m++)
            u[m * T] = cscale(mul_ipow(m, v[tri(k, m) * T]), m ? 2.0 : 1.0);
        fold_apply(Dn, k, u, x, T, false);
        double2 pb = make_double2(1.0, 0.0);
        for (int j = 0; j <= k; j++) {
            x[j * T] = cscale(cmul(x[j * T], pb), j ? 2.0 : 1.0);
            pb = cmul(pb, eb_);
        }
        fold_apply(Dn, k, x, u, T, true);
        double2 ph = make_double2(1.0, 0.0);
        for (int l = 0; l <= k; l++) {
            const int c = tri(k, l);
            const double2 r = cscale(cmul(mul_ipow(4 - (l & 3), u[l * T]), ph), Ft[c]);
            const double rx = seg_sum(r.x, same), ry = seg_sum(r.y, same);
            if (head) {
                atomicAdd(&L[gt * nc + c].x, rx);
                atomicAdd(&L[gt * nc + c].y, ry);
            }
            ph = cmul(ph, ea);
        }
        Dn += (k + 1) * (k + 1);
    }
}

// ---------------------------------------------------------------------------
// M2M and L2L in the rotational form (double precision). L2L: rotate the parent's local
// expansion onto the child offset, translate along z, rotate back:
//   local, rotated frame (Lt = L / F):    Lt'_j^i = sum_{k>=j} Lt_k^i F_ki rho^{k-j}/(k-j)! / F_ji
// The forward rotation of a local expansion uses the two folds of the M2L
// back rotation with conjugate phases.
// ---------------------------------------------------------------------------

// One warp per child box. Every stage (phase, fold, axial shift) is
// independent across degrees, so the warp's lanes take the outputs of all
// degrees at once (coefficient c = lane, lane + 32, ...) and the child's
// vectors sit in the warp's slice of shared memory between the stages:
//   multipole, rotated frame (Mt = F M):  Mt'_n^m = F_nm sum_k rho^k/k! Mt_{n-k}^m / F_{n-k,m}
//   local, rotated frame (Lt = L / F):   Lt'_j^i = sum_{k>=j} Lt_k^i F_ki rho^{k-j}/(k-j)! / F_ji
// GB300 retires about two FP64 multiply-adds per clock per SM, so a child
// spread over a warp keeps each lane's serial chain to a few dozen
// operations (the small levels near the root finish in microseconds), and
// blocks of 1 to 8 warps spread even a small level over all SMs.
__device__ __forceinline__ int degree_of(int c) {
    int n = (int)((sqrtf(8.f * (float)c + 1.f) - 1.f) * 0.5f);
    while (tri(n + 1, 0) <= c) n++;
    while (n > 0 && tri(n, 0) > c) n--;
    return n;
}

// One warp per box: lane n <= p forms r^-n (a single division), and each
// coefficient takes its degree's factor from that lane.
__device__ __forceinline__ double inv_radius_pow(const double *__restrict__ radius, int64_t g, int p, int lane) {
    double pw = 1.0;
    if (lane <= p) {
        const double r = radius[g] > 0.0 ? radius[g] : 1.0;
        double b = 1.0 / r;
        for (int e = lane; e; e >>= 1) {
            if (e & 1) pw *= b;
            b *= b;
        }
    }
    return pw;
}

// Box g's coefficients times r^-n, by one warp: Mhat = M / r^n into Mf
// (float, read through L2: completed by other warps of the launch) or
// L = Lhat / r^n into L.
__device__ __forceinline__ void warp_scale_multipole(const double *__restrict__ radius, int64_t g, int p,
                                                     const double2 *M, float2 *Mf) {
    const int nc = ncoef(p), lane = threadIdx.x & 31;
    const double pw = inv_radius_pow(radius, g, p, lane);
    for (int c0 = 0; c0 < nc; c0 += 32) {  // warp-uniform trip count around the shuffle
        const int c = c0 + lane;
        const double sc = __shfl_sync(0xffffffffu, pw, degree_of(min(c, nc - 1)));
        if (c < nc) {
            const double2 m = __ldcg(M + g * nc + c);
            Mf[g * mf_stride(p) + c] = make_float2((float)(m.x * sc), (float)(m.y * sc));
        }
    }
}

__device__ __forceinline__ void warp_unscale_local(const double *__restrict__ radius, int64_t g, int p,
                                                   const double2 *__restrict__ Lh, double2 *L) {
    const int nc = ncoef(p), lane = threadIdx.x & 31;
    const double pw = inv_radius_pow(radius, g, p, lane);
    for (int c0 = 0; c0 < nc; c0 += 32) {
        const int c = c0 + lane;
        const double sc = __shfl_sync(0xffffffffu, pw, degree_of(min(c, nc - 1)));
        if (c < nc) {
            const double2 h = Lh[g * nc + c];
            L[g * nc + c] = make_double2(h.x * sc, h.y * sc);
        }
    }
    __syncwarp();
}

// double2 slots of one warp's slice: A, B (nc each), powers of e^{ia} and
// e^{ib} (p+1 each), rho^k/k! (p+1 doubles)
__host__ __device__ inline int warp_slice(int p) { return 2 * ncoef(p) + 2 * (p + 1) + (p + 2) / 2; }
// doubles of the shared tables: D, F, 1/F, 1/k
__host__ __device__ inline int warp_tabs(int p) {
    return (p + 1) * (p + 2) * (2 * p + 3) / 6 + 2 * ncoef(p) + p + 2;
}

// post(c, k, out_k) for out_k = fold(D^n) of in (degree n of c, k = c - tri(n, 0))
template <bool kTranspose, typename Post>
__device__ __forceinline__ void fold_all(const double *__restrict__ Dt, int nc, const double2 *in, int lane,
                                         Post post) {
    for (int c = lane; c < nc; c += 32) {
        const int n = degree_of(c), b = tri(n, 0), k = c - b, par = (n + k) & 1;
        const double *Dn = Dt + n * (n + 1) * (2 * n + 1) / 6;
        double ev = 0.0, od = 0.0;  // sums over even and odd m
        int m = 0;
        for (; m + 1 <= n; m += 2) {
            const double2 v0 = in[b + m], v1 = in[b + m + 1];
            ev = fma(kTranspose ? Dn[m * (n + 1) + k] : Dn[k * (n + 1) + m], par ? v0.y : v0.x, ev);
            od = fma(kTranspose ? Dn[(m + 1) * (n + 1) + k] : Dn[k * (n + 1) + m + 1], par ? v1.x : v1.y, od);
        }
        if (m == n) {
            const double2 v0 = in[b + m];
            ev = fma(kTranspose ? Dn[m * (n + 1) + k] : Dn[k * (n + 1) + m], par ? v0.y : v0.x, ev);
        }
        post(c, k, par ? make_double2(od, ev) : make_double2(ev, od));
    }
}

struct WarpChild {
    double2 *A, *B, *pa, *pb;
    double *f;
    const double *Dt, *Ft, *iFt;
    int64_t gc, gp;
    int nc, lane;
};

// Tables into shared memory (every thread of the block; one barrier).
__device__ __forceinline__ double *stage_child_tables(int p, const double *__restrict__ gtab, double2 *sw) {
    const int nc = ncoef(p), nw = blockDim.x >> 5;
    const int nD = (p + 1) * (p + 2) * (2 * p + 3) / 6;
    double *tab = (double *)(sw + nw * warp_slice(p));
    for (int i = threadIdx.x; i < nD; i += blockDim.x) tab[i] = gtab[i];
    for (int i = threadIdx.x; i < 2 * nc + p + 2; i += blockDim.x) tab[nD + i] = gtab[2 * nD + i];
    __syncthreads();
    return tab;
}

// The warp's child gc, its parent gp, and the powers of the child-to-parent
// offset, in the warp's slice of shared memory (warp-synchronous only).
// the child-to-parent offset's powers e^{ia}, e^{ib} and rho^k/k! (lanes
// 0..2) into the warp's slice
__device__ __forceinline__ void warp_child_geometry(WarpChild &W, int p, const double *__restrict__ centre) {
    const int64_t gc = W.gc, gp = W.gp;
    const int lane = W.lane;
    __syncwarp();
    if (lane < 3) {
        const double dx = centre[3 * gc] - centre[3 * gp], dy = centre[3 * gc + 1] - centre[3 * gp + 1],
                     dz = centre[3 * gc + 2] - centre[3 * gp + 2];
        const double rxy = sqrt(dx * dx + dy * dy), rho = sqrt(dx * dx + dy * dy + dz * dz);
        if (lane == 2) {
            const double *ik = W.iFt + W.nc;
            double t = 1.0;
            for (int k = 0; k <= p; k++) {
                W.f[k] = t;
                t = t * rho * ik[k + 1];
            }
        } else {
            double2 z;
            if (lane == 0) {
                const double irxy = rxy > 0.0 ? 1.0 / rxy : 0.0;
                z = rxy > 0.0 ? make_double2(dx * irxy, dy * irxy) : make_double2(1.0, 0.0);
            } else {
                const double irho = rho > 0.0 ? 1.0 / rho : 0.0;
                z = rho > 0.0 ? make_double2(dz * irho, rxy * irho) : make_double2(1.0, 0.0);
            }
            double2 *pw = lane == 0 ? W.pa : W.pb, t = make_double2(1.0, 0.0);
            for (int k = 0; k <= p; k++) {
                pw[k] = t;
                t = cmul(t, z);
            }
        }
    }
    __syncwarp();
}

// The warp's child gc, its parent gp, and the powers of the child-to-parent
// offset, in the warp's slice of shared memory (warp-synchronous only).
__device__ __forceinline__ void warp_child_init(int64_t gc, int64_t gp, int p, const double *__restrict__ centre,
                                                const double *tab, double2 *sw, WarpChild &W) {
    const int nc = ncoef(p), w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nD = (p + 1) * (p + 2) * (2 * p + 3) / 6;
    W.A = sw + w * warp_slice(p);
    W.B = W.A + nc;
    W.pa = W.B + nc;
    W.pb = W.pa + p + 1;
    W.f = (double *)(W.pb + p + 1);
    W.Dt = tab;
    W.Ft = tab + nD;
    W.iFt = W.Ft + nc;
    W.gc = gc;
    W.gp = gp;
    W.nc = nc;
    W.lane = lane;
    warp_child_geometry(W, p, centre);
}

// M2M of the warp's child into its parent (atomic adds). The child's
// multipole is read through L2: in the one-launch upward pass another warp
// completed it.
__device__ __forceinline__ void m2m_body(const WarpChild &W, double2 *M) {
    const int nc = W.nc, lane = W.lane;
    double2 *A = W.A, *B = W.B;
    const double2 *pa = W.pa, *pb = W.pb;
    const double *f = W.f, *Ft = W.Ft, *iFt = W.iFt;
    // forward rotation: u = F M (-i e^{ia})^m, doubled for m > 0
    for (int c = lane; c < nc; c += 32) {
        const int m = c - tri(degree_of(c), 0);
        A[c] = cscale(cmul(__ldcg(M + W.gc * nc + c), mul_ipow(4 - (m & 3), pa[m])), Ft[c] * (m ? 2.0 : 1.0));
    }
    __syncwarp();
    fold_all<false>(W.Dt, nc, A, lane,
                    [&](int c, int k, double2 r) { B[c] = cscale(cmul(r, pb[k]), k ? 2.0 : 1.0); });
    __syncwarp();
    // v = i^m (folded back); the axial input is v / F
    fold_all<true>(W.Dt, nc, B, lane, [&](int c, int m, double2 r) { A[c] = cscale(mul_ipow(m, r), iFt[c]); });
    __syncwarp();
    // axial shift; then the back rotation's i^-m and doubling
    for (int c = lane; c < nc; c += 32) {
        const int n = degree_of(c), m = c - tri(n, 0);
        double re = 0.0, im = 0.0;
        for (int k = 0; k <= n - m; k++) {
            const double2 t = A[tri(n - k, m)];
            re = fma(f[k], t.x, re);
            im = fma(f[k], t.y, im);
        }
        B[c] = cscale(mul_ipow(4 - (m & 3), make_double2(re, im)), Ft[c] * (m ? 2.0 : 1.0));
    }
    __syncwarp();
    fold_all<false>(W.Dt, nc, B, lane,
                    [&](int c, int k, double2 r) { A[c] = cscale(cmul(r, cconj(pb[k])), k ? 2.0 : 1.0); });
    __syncwarp();
    double2 *Mp = M + W.gp * nc;
    fold_all<true>(W.Dt, nc, A, lane, [&](int c, int m, double2 r) {
        const double2 t = cscale(cmul(mul_ipow(m, r), cconj(pa[m])), iFt[c]);
        atomicAdd(&Mp[c].x, t.x);
        atomicAdd(&Mp[c].y, t.y);
    });
    __syncwarp();
}

// L2L of the warp's parent into its child (added to the child's local
// expansion). The parent's expansion is read through L2: in the one-launch
// downward pass another warp completed it.
__device__ __forceinline__ void l2l_body(const WarpChild &W, double2 *L, int pmax) {
    const int nc = W.nc, lane = W.lane;
    double2 *A = W.A, *B = W.B;
    const double2 *pa = W.pa, *pb = W.pb;
    const double *f = W.f, *Ft = W.Ft, *iFt = W.iFt;
    // forward rotation of the parent's local expansion: Lt = L / F, i^l e^{-ila}, doubled for l > 0
    for (int c = lane; c < nc; c += 32) {
        const int l = c - tri(degree_of(c), 0);
        A[c] = cscale(cmul(mul_ipow(l, __ldcg(L + W.gp * nc + c)), cconj(pa[l])), (l ? 2.0 : 1.0) * iFt[c]);
    }
    __syncwarp();
    fold_all<false>(W.Dt, nc, A, lane,
                    [&](int c, int k, double2 r) { B[c] = cscale(cmul(r, cconj(pb[k])), k ? 2.0 : 1.0); });
    __syncwarp();
    // v = i^-m (folded back); the axial input is v F
    fold_all<true>(W.Dt, nc, B, lane,
                   [&](int c, int m, double2 r) { A[c] = cscale(mul_ipow(4 - (m & 3), r), Ft[c]); });
    __syncwarp();
    // axial shift; then the back rotation's i^m and doubling
    for (int c = lane; c < nc; c += 32) {
        const int j = degree_of(c), i = c - tri(j, 0);
        double re = 0.0, im = 0.0;
        for (int k = j; k <= pmax; k++) {
            const double2 t = A[tri(k, i)];
            re = fma(f[k - j], t.x, re);
            im = fma(f[k - j], t.y, im);
        }
        B[c] = cscale(mul_ipow(i, make_double2(re, im)), iFt[c] * (i ? 2.0 : 1.0));
    }
    __syncwarp();
    fold_all<false>(W.Dt, nc, B, lane,
                    [&](int c, int k, double2 r) { A[c] = cscale(cmul(r, pb[k]), k ? 2.0 : 1.0); });
    __syncwarp();
    double2 *Lc = L + W.gc * nc;
    fold_all<true>(W.Dt, nc, A, lane, [&](int c, int l, double2 r) {
        Lc[c] = cadd(Lc[c], cscale(cmul(mul_ipow(4 - (l & 3), r), pa[l]), Ft[c]));
    });
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Double-float translations (mixed form). GB300's FP64 pipe retires ~1.7
// multiply-adds per clock per SM against 128 on the FP32 pipe, so M2M and
// L2L in double precision cost as much as all the single-precision stages
// together. The mixed form runs them in double-float arithmetic instead: a
// value is an unevaluated sum hi + lo of two floats (Dekker's and Knuth's
// error-free transformations: TwoSum, and TwoProd through the fused
// multiply-add), about 44 significant bits, every operation an explicitly
// rounded intrinsic so that the compiler neither contracts nor reorders it.
// Float's exponent range would not hold a deep box's high-degree
// multipole (M_n ~ q r^n), so the coefficients are scaled while translated
// by s = 2^e, the power of two within a factor 2 below the parent's radius
// (exact in double): M2M reads M_n / s^n and writes s^n times its result,
// L2L reads L_n s^n and writes s^-n times its result, and the axial factors
// become (rho / s)^k / k!: every value stays O(1). Rotations act within a
// degree and commute with the scaling. The stored expansions stay double.
// ---------------------------------------------------------------------------
struct DF {
    float h, l;
};
struct CDF {
    DF x, y;
};
__device__ __forceinline__ DF df_of(double d) {
    const float h = __double2float_rn(d);
    return {h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double df_val(DF a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ DF df_neg(DF a) { return {-a.h, -a.l}; }
// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
// renormalise (|a| >= |b|, or a + b rounds to a)
__device__ __forceinline__ DF df_fast(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// a b: the product's rounding error from the fused multiply-add, plus the cross terms
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return df_fast(p, e);
}
// a b + c
__device__ __forceinline__ DF df_fma(DF a, DF b, DF c) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const DF s = df_two_sum(p, c.h);
    return df_fast(s.h, __fadd_rn(s.l, __fadd_rn(e, c.l)));
}
__device__ __forceinline__ CDF cdf_of(double2 v) { return {df_of(v.x), df_of(v.y)}; }
__device__ __forceinline__ double2 cdf_val(CDF a) { return make_double2(df_val(a.x), df_val(a.y)); }
__device__ __forceinline__ CDF cdf_conj(CDF a) { return {a.x, df_neg(a.y)}; }
__device__ __forceinline__ CDF cdf_mul(CDF a, CDF b) {
    return {df_fma(a.x, b.x, df_neg(df_mul(a.y, b.y))), df_fma(a.x, b.y, df_mul(a.y, b.x))};
}
__device__ __forceinline__ CDF cdf_scale(CDF a, DF s) { return {df_mul(a.x, s), df_mul(a.y, s)}; }
// exact doubling
__device__ __forceinline__ CDF cdf_twice(CDF a) {
    return {{2.f * a.x.h, 2.f * a.x.l}, {2.f * a.y.h, 2.f * a.y.l}};
}
__device__ __forceinline__ CDF cdf_ipow(int m, CDF v) {  // i^m v
    switch (m & 3) {
        case 0: return v;
        case 1: return {df_neg(v.y), v.x};
        case 2: return {df_neg(v.x), df_neg(v.y)};
        default: return {v.y, df_neg(v.x)};
    }
}

// Geometry of box g's translation to / from its parent, formed once per
// plan in double (k_box_geo) and kept as double-float pairs: the unit
// complex numbers e^{ia} (azimuth) and e^{ib} (polar angle of the offset),
// and q = rho / s for the scale s = 2^e, the power of two with
// s <= r_p < 2 s (r_p the parent's radius): scaling by powers of two is exact
// and needs no power of r_p in float, whose range r_p^12 of a deep box
// would leave.
struct alignas(16) BoxGeo {
    CDF za, zb;
    DF q;
    int e;     // s = 2^e
    int skip;  // an empty box outside its parent's box (rho > 2 r_p): nothing to translate
};



// 1/k! as double-float pairs, built at compile time
struct IFact {
    DF v[FMM_MAX_P + 2];
};
constexpr IFact make_ifact() {
    IFact t{};
    double f = 1.0;
    for (int k = 0; k <= FMM_MAX_P + 1; k++) {
        if (k > 1) f /= (double)k;
        const float h = (float)f;
        t.v[k] = DF{h, (float)(f - (double)h)};
    }
    return t;
}
__constant__ IFact c_ifact = make_ifact();

__device__ __forceinline__ DF df_pow(DF x, int k) {
    DF r = {1.f, 0.f};
    while (k) {
        if (k & 1) r = df_mul(r, x);
        k >>= 1;
        if (k) x = df_mul(x, x);
    }
    return r;
}
__device__ __forceinline__ CDF cdf_pow(CDF z, int k) {
    CDF r = {{1.f, 0.f}, {0.f, 0.f}};
    while (k) {
        if (k & 1) r = cdf_mul(r, z);
        k >>= 1;
        if (k) z = cdf_mul(z, z);
    }
    return r;
}

// one thread per box (box 0 has no parent)
__global__ void k_box_geo(int64_t nbox, int step, const double *__restrict__ centre,
                          const double *__restrict__ radius, BoxGeo *__restrict__ geo) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nbox; g += (int64_t)gridDim.x * blockDim.x) {
        BoxGeo o{};
        if (g == 0) {
            o.skip = 1;
            geo[g] = o;
            continue;
        }
        const int64_t gp = ((g + 1) >> step) - 1;
        const double dx = centre[3 * g] - centre[3 * gp], dy = centre[3 * g + 1] - centre[3 * gp + 1],
                     dz = centre[3 * g + 2] - centre[3 * gp + 2];
        const double rxy = sqrt(dx * dx + dy * dy), rho = sqrt(dx * dx + dy * dy + dz * dz);
        const double rp = radius[gp] > 0.0 ? radius[gp] : 1.0;
        // s = 2^e <= r_p < 2^(e+1); |e| <= 48 keeps s^n within double range for n <= 20
        const int e = max(-48, min(48, ilogb(rp)));
        o.za = rxy > 0.0 ? cdf_of(make_double2(dx / rxy, dy / rxy)) : cdf_of(make_double2(1.0, 0.0));
        o.zb = rho > 0.0 ? cdf_of(make_double2(dz / rho, rxy / rho)) : cdf_of(make_double2(1.0, 0.0));
        o.q = df_of(rho * pow2i(-e));
        o.e = e;
        o.skip = rho > 2.0 * rp;
        geo[g] = o;
    }
}

struct WarpChildDF {
    CDF *A, *B, *pa, *pb;
    DF *f;  // (rho / s)^k / k!
    const DF *Dt, *Ft, *iFt;
    int64_t gc, gp;
    int nc, lane, e;  // s = 2^e
    bool skip;
};

// The double-float tables into shared memory (plain copies; same offsets as the double tables)
__device__ __forceinline__ const DF *stage_child_tables_df(int p, const float2 *__restrict__ gtab, double2 *sw) {
    const int nc = ncoef(p), nw = blockDim.x >> 5;
    const int nD = (p + 1) * (p + 2) * (2 * p + 3) / 6;
    float2 *tab = (float2 *)(sw + nw * warp_slice(p));
    for (int i = threadIdx.x; i < nD; i += blockDim.x) tab[i] = gtab[i];
    for (int i = threadIdx.x; i < 2 * nc + p + 2; i += blockDim.x) tab[nD + i] = gtab[2 * nD + i];
    __syncthreads();
    return (const DF *)tab;
}

// the warp's child: the powers of its geometry, lanes over the degrees, all
// in double-float on the FP32 pipe
__device__ __forceinline__ void warp_child_init_df(int64_t gc, int64_t gp, int p, const BoxGeo *__restrict__ geo,
                                                   const DF *tab, double2 *sw, WarpChildDF &W) {
    const int nc = ncoef(p), w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nD = (p + 1) * (p + 2) * (2 * p + 3) / 6;
    double2 *base = sw + w * warp_slice(p);
    W.A = (CDF *)base;
    W.B = W.A + nc;
    W.pa = W.B + nc;
    W.pb = W.pa + p + 1;
    W.f = (DF *)(W.pb + p + 1);
    W.Dt = tab;
    W.Ft = tab + nD;
    W.iFt = W.Ft + nc;
    W.gc = gc;
    W.gp = gp;
    W.nc = nc;
    W.lane = lane;
    const BoxGeo o = geo[gc];
    W.skip = o.skip != 0;
    W.e = o.e;
    __syncwarp();
    for (int k = lane; k <= p; k += 32) {
        W.pa[k] = cdf_pow(o.za, k);
        W.pb[k] = cdf_pow(o.zb, k);
        W.f[k] = df_mul(df_pow(o.q, k), c_ifact.v[k]);
    }
    __syncwarp();
}

// out_k = fold(D^n) of in, in double-float (as fold_all)
template <bool kTranspose, typename Post>
__device__ __forceinline__ void fold_all_df(const DF *__restrict__ Dt, int nc, const CDF *in, int lane, Post post) {
    for (int c = lane; c < nc; c += 32) {
        const int n = degree_of(c), b = tri(n, 0), k = c - b, par = (n + k) & 1;
        const DF *Dn = Dt + n * (n + 1) * (2 * n + 1) / 6;
        DF ev = {0.f, 0.f}, od = {0.f, 0.f};  // sums over even and odd m
        int m = 0;
        for (; m + 1 <= n; m += 2) {
            const CDF v0 = in[b + m], v1 = in[b + m + 1];
            ev = df_fma(kTranspose ? Dn[m * (n + 1) + k] : Dn[k * (n + 1) + m], par ? v0.y : v0.x, ev);
            od = df_fma(kTranspose ? Dn[(m + 1) * (n + 1) + k] : Dn[k * (n + 1) + m + 1], par ? v1.x : v1.y, od);
        }
        if (m == n) {
            const CDF v0 = in[b + m];
            ev = df_fma(kTranspose ? Dn[m * (n + 1) + k] : Dn[k * (n + 1) + m], par ? v0.y : v0.x, ev);
        }
        post(c, k, par ? CDF{od, ev} : CDF{ev, od});
    }
}

// m2m_body in double-float on scaled coefficients
__device__ __forceinline__ void m2m_body_df(const WarpChildDF &W, double2 *M) {
    const int nc = W.nc, lane = W.lane;
    CDF *A = W.A, *B = W.B;
    const CDF *pa = W.pa, *pb = W.pb;
    const DF *f = W.f, *Ft = W.Ft, *iFt = W.iFt;
    for (int c = lane; c < nc; c += 32) {
        const int n = degree_of(c), m = c - tri(n, 0);
        const double sc = pow2i(-W.e * n);  // M_n / s^n, exact
        const double2 v = __ldcg(M + W.gc * nc + c);
        const CDF u = cdf_mul(cdf_of(make_double2(v.x * sc, v.y * sc)), cdf_ipow(4 - (m & 3), pa[m]));
        A[c] = m ? cdf_twice(cdf_scale(u, Ft[c])) : cdf_scale(u, Ft[c]);
    }
    __syncwarp();
    fold_all_df<false>(W.Dt, nc, A, lane, [&](int c, int k, CDF r) {
        const CDF t = cdf_mul(r, pb[k]);
        B[c] = k ? cdf_twice(t) : t;
    });
    __syncwarp();
    fold_all_df<true>(W.Dt, nc, B, lane, [&](int c, int m, CDF r) { A[c] = cdf_scale(cdf_ipow(m, r), iFt[c]); });
    __syncwarp();
    for (int c = lane; c < nc; c += 32) {
        const int n = degree_of(c), m = c - tri(n, 0);
        DF re = {0.f, 0.f}, im = {0.f, 0.f};
        for (int k = 0; k <= n - m; k++) {
            const CDF t = A[tri(n - k, m)];
            re = df_fma(f[k], t.x, re);
            im = df_fma(f[k], t.y, im);
        }
        const CDF u = cdf_scale(cdf_ipow(4 - (m & 3), CDF{re, im}), Ft[c]);
        B[c] = m ? cdf_twice(u) : u;
    }
    __syncwarp();
    fold_all_df<false>(W.Dt, nc, B, lane, [&](int c, int k, CDF r) {
        const CDF t = cdf_mul(r, cdf_conj(pb[k]));
        A[c] = k ? cdf_twice(t) : t;
    });
    __syncwarp();
    double2 *Mp = M + W.gp * nc;
    fold_all_df<true>(W.Dt, nc, A, lane, [&](int c, int m, CDF r) {
        const double2 t = cdf_val(cdf_scale(cdf_mul(cdf_ipow(m, r), cdf_conj(pa[m])), iFt[c]));
        const double sc = pow2i(W.e * degree_of(c));  // times s^n, exact
        atomicAdd(&Mp[c].x, t.x * sc);
        atomicAdd(&Mp[c].y, t.y * sc);
    });
    __syncwarp();
}

// l2l_body in double-float on scaled coefficients
__device__ __forceinline__ void l2l_body_df(const WarpChildDF &W, double2 *L, int pmax) {
    const int nc = W.nc, lane = W.lane;
    CDF *A = W.A, *B = W.B;
    const CDF *pa = W.pa, *pb = W.pb;
    const DF *f = W.f, *Ft = W.Ft, *iFt = W.iFt;
    for (int c = lane; c < nc; c += 32) {
        const int n = degree_of(c), l = c - tri(n, 0);
        const double sc = pow2i(W.e * n);  // L_n s^n, exact
        const double2 w = __ldcg(L + W.gp * nc + c);
        const CDF v = cdf_of(make_double2(w.x * sc, w.y * sc));
        const CDF u = cdf_scale(cdf_mul(cdf_ipow(l, v), cdf_conj(pa[l])), iFt[c]);
        A[c] = l ? cdf_twice(u) : u;
    }
    __syncwarp();
    fold_all_df<false>(W.Dt, nc, A, lane, [&](int c, int k, CDF r) {
        const CDF t = cdf_mul(r, cdf_conj(pb[k]));
        B[c] = k ? cdf_twice(t) : t;
    });
    __syncwarp();
    fold_all_df<true>(W.Dt, nc, B, lane,
                      [&](int c, int m, CDF r) { A[c] = cdf_scale(cdf_ipow(4 - (m & 3), r), Ft[c]); });
    __syncwarp();
    for (int c = lane; c < nc; c += 32) {
        const int j = degree_of(c), i = c - tri(j, 0);
        DF re = {0.f, 0.f}, im = {0.f, 0.f};
        for (int k = j; k <= pmax; k++) {
            const CDF t = A[tri(k, i)];
            re = df_fma(f[k - j], t.x, re);
            im = df_fma(f[k - j], t.y, im);
        }
        const CDF u = cdf_scale(cdf_ipow(i, CDF{re, im}), iFt[c]);
        B[c] = i ? cdf_twice(u) : u;
    }
    __syncwarp();
    fold_all_df<false>(W.Dt, nc, B, lane, [&](int c, int k, CDF r) {
        const CDF t = cdf_mul(r, pb[k]);
        A[c] = k ? cdf_twice(t) : t;
    });
    __syncwarp();
    double2 *Lc = L + W.gc * nc;
    fold_all_df<true>(W.Dt, nc, A, lane, [&](int c, int l, CDF r) {
        const double2 t = cdf_val(cdf_scale(cdf_mul(cdf_ipow(4 - (l & 3), r), pa[l]), Ft[c]));
        const double sc = pow2i(-W.e * degree_of(c));  // times s^-n, exact
        Lc[c] = cadd(Lc[c], make_double2(t.x * sc, t.y * sc));
    });
    __syncwarp();
}

// What the translation kernels read besides the expansions.
struct TrIn {
    const double *centre, *radius;
    const BoxGeo *geo;      // double-float translations
    const double *tab;      // tables in double (global memory)
    const float2 *tab_df;   // the same as double-float pairs
};

// One translation of child gc with parent gp, in double (FP64 form) or in
// double-float (DFT: mixed form); `tab` from stage_tables<DFT>.
template <bool DFT>
__device__ __forceinline__ const void *stage_tables(int p, const TrIn &a, double2 *sw) {
    if constexpr (DFT)
        return stage_child_tables_df(p, a.tab_df, sw);
    else
        return stage_child_tables(p, a.tab, sw);
}
template <bool DFT>
__device__ __forceinline__ void m2m_one(int64_t gc, int64_t gp, int p, const TrIn &a, double2 *M, const void *tab,
                                        double2 *sw) {
    if constexpr (DFT) {
        WarpChildDF W;
        warp_child_init_df(gc, gp, p, a.geo, (const DF *)tab, sw, W);
        if (!W.skip) m2m_body_df(W, M);  // skipped: an empty child, whose multipole is zero
    } else {
        WarpChild W;
        warp_child_init(gc, gp, p, a.centre, (const double *)tab, sw, W);
        m2m_body(W, M);
    }
}
template <bool DFT>
__device__ __forceinline__ void l2l_one(int64_t gc, int64_t gp, int p, const TrIn &a, double2 *L, const void *tab,
                                        double2 *sw) {
    if constexpr (DFT) {
        WarpChildDF W;
        warp_child_init_df(gc, gp, p, a.geo, (const DF *)tab, sw, W);
        if (!W.skip) {
            l2l_body_df(W, L, p);
        } else {
            // an empty box outside its parent's (tight) box: its expansion
            // reaches no point, and translated that far it would leave the
            // float range; formed in double with the tables from global memory
            const int nD = (p + 1) * (p + 2) * (2 * p + 3) / 6;
            WarpChild V;
            V.A = (double2 *)W.A;
            V.B = (double2 *)W.B;
            V.pa = (double2 *)W.pa;
            V.pb = (double2 *)W.pb;
            V.f = (double *)W.f;
            V.Dt = a.tab;
            V.Ft = a.tab + 2 * nD;
            V.iFt = V.Ft + W.nc;
            V.gc = gc;
            V.gp = gp;
            V.nc = W.nc;
            V.lane = W.lane;
            warp_child_geometry(V, p, a.centre);
            l2l_body(V, L, p);
        }
    } else {
        WarpChild W;
        warp_child_init(gc, gp, p, a.centre, (const double *)tab, sw, W);
        l2l_body(W, L, p);
    }
}

template <bool DFT>
__global__ void __launch_bounds__(kWarpChildMax * 32)
k_m2m_warp(int level, int step, int p, TrIn a, double2 *M) {
    extern __shared__ double2 sw[];
    const void *tab = stage_tables<DFT>(p, a, sw);
    const int64_t j = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= ((int64_t)1 << level)) return;  // no block barrier follows
    const int64_t gc = ((int64_t)1 << level) - 1 + j;
    m2m_one<DFT>(gc, ((gc + 1) >> step) - 1, p, a, M, tab, sw);
}

template <bool DFT>
__global__ void __launch_bounds__(kWarpChildMax * 32)
k_l2l_warp(int level, int step, int p, TrIn a, double2 *L) {
    extern __shared__ double2 sw[];
    const void *tab = stage_tables<DFT>(p, a, sw);
    const int64_t j = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= ((int64_t)1 << level)) return;
    const int64_t gc = ((int64_t)1 << level) - 1 + j;
    l2l_one<DFT>(gc, ((gc + 1) >> step) - 1, p, a, L, tab, sw);
}

// Leaf j's walk up: translate into the parent; the warp that delivers a
// parent's second child (an arrival counter per parent) carries on with that
// parent, whose multipole is then complete, so no warp ever waits.
// Translations stop at level `stop` (no multipole above it is read). With
// `Mf`, each box the walk completes (its leaf, every parent it carries on,
// down to level `stop`) is also scaled into Mf for the single-precision M2L.
template <bool DFT>
__device__ __forceinline__ void m2m_walk(int B, int stop, int64_t j, int p, const TrIn &a, double2 *M, float2 *Mf,
                                         const void *tab, double2 *sw, unsigned *arrive) {
    const int lane = threadIdx.x & 31;
    int64_t gc = ((int64_t)1 << B) - 1 + j;
    for (int l = B;; l--) {
        if (Mf) warp_scale_multipole(a.radius, gc, p, M, Mf);
        if (l <= stop) break;
        const int64_t gp = (gc - 1) >> 1;
        m2m_one<DFT>(gc, gp, p, a, M, tab, sw);
        __threadfence();
        unsigned old = 0;
        if (lane == 0) old = atomicAdd(&arrive[gp], 1u);
        old = __shfl_sync(0xffffffffu, old, 0);
        if (old == 0) break;  // the sibling is still on its way: it carries the parent on
        __threadfence();
        gc = gp;
    }
}

// The whole upward pass (binary levels) in one launch, one warp per leaf.
template <bool DFT>
__global__ void __launch_bounds__(kWarpChildMax * 32)
k_m2m_up(int B, int stop, int p, TrIn a, double2 *M, unsigned *arrive) {
    extern __shared__ double2 sw[];
    const void *tab = stage_tables<DFT>(p, a, sw);
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
    const int64_t nleaf = (int64_t)1 << B;
    for (int64_t j = blockIdx.x * (int64_t)nw + w; j < nleaf; j += (int64_t)gridDim.x * nw)
        m2m_walk<DFT>(B, stop, j, p, a, M, nullptr, tab, sw, arrive);
}

// batched: blocks of kWarpChildMax leaves of one system each; every box the
// walks complete is scaled for the single-precision M2L on the way
__global__ void __launch_bounds__(kWarpChildMax * 32)
k_b_m2m_up(const BatchSys *__restrict__ S, const int32_t *__restrict__ off, int nsys, int p,
           const float2 *__restrict__ tab_df) {
    extern __shared__ double2 sw[];
    const DF *tab = stage_child_tables_df(p, tab_df, sw);
    const int s = batch_sys_of(off, nsys, blockIdx.x);
    const BatchSys &y = S[s];
    const TrIn a{y.centre, y.radius, (const BoxGeo *)y.box_geo, nullptr, tab_df};
    const int64_t j = (blockIdx.x - off[s]) * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j < y.nleaf) m2m_walk<true>(y.B, min(y.lw, y.B), j, p, a, y.M, y.Mf, tab, sw, y.arrive);
}

// The whole downward pass (binary levels) in one launch: warps take boxes in
// chunks of kL2LChunk from one counter in heap order (level by level), so a
// box's parent was taken earlier by a running warp; a box whose parent holds
// a local expansion (parent level >= lw) waits for the parent's flag, then
// adds the parent's L2L to its own expansion and raises its flag. Each wait
// is bounded (wait_limit sleeps of ~0.1 us): a wait that runs out sets bit
// 16 of err[1] (FMM_ETIMEDOUT, results invalid) and the box goes on.
// `withhold` (>= 0: tests only) is a box whose flag is never raised. With
// `Lh`, a box first takes its own M2L result L = Lhat / r^n (the
// single-precision M2L's output), then its parent's L2L.
constexpr int kL2LChunk = 8;
template <bool DFT>
__device__ __forceinline__ void l2l_chunk(int lw, int p, const TrIn &a, const double2 *__restrict__ Lh, double2 *L,
                                          const void *tab, double2 *sw, int *done, int *err, int64_t g0, int64_t g1,
                                          long long wait_limit, long long withhold) {
    const int lane = threadIdx.x & 31;
    for (int64_t g = g0; g < g1; g++) {
        const int l = 63 - __clzll((unsigned long long)(g + 1));
        const int64_t gp = (g - 1) >> 1;
        if (Lh) warp_unscale_local(a.radius, g, p, Lh, L);
        if (l - 1 >= lw) {
            if (gp > 0) {  // the root's expansion is complete before the launch
                int ok = 1;
                if (lane == 0) {
                    long long it = 0;
                    while (__ldcg(done + gp) == 0) {
                        if (++it > wait_limit) {
                            ok = 0;
                            atomicOr(err + 1, 16);
                            break;
                        }
                        __nanosleep(100);
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                (void)ok;  // a box whose wait ran out goes on: the error word says the results are invalid
                __threadfence();  // the parent's expansion after its flag
            }
            l2l_one<DFT>(g, gp, p, a, L, tab, sw);
            __threadfence();
        }
        if (lane == 0 && g != withhold) atomicExch(done + g, 1);
        __syncwarp();
    }
}

template <bool DFT>
__global__ void __launch_bounds__(kWarpChildMax * 32)
k_l2l_down(int B, int lw, int p, TrIn a, double2 *L, int *done, unsigned long long *next, int *err,
           long long wait_limit, long long withhold) {
    extern __shared__ double2 sw[];
    const void *tab = stage_tables<DFT>(p, a, sw);
    const int lane = threadIdx.x & 31;
    const int64_t nbox = ((int64_t)2 << B) - 1;
    for (;;) {
        unsigned long long c0 = 0;
        if (lane == 0) c0 = atomicAdd(next, (unsigned long long)kL2LChunk);
        c0 = __shfl_sync(0xffffffffu, c0, 0);
        if ((int64_t)c0 + 1 >= nbox) break;
        l2l_chunk<DFT>(lw, p, a, nullptr, L, tab, sw, done, err, (int64_t)c0 + 1,
                       std::min<int64_t>((int64_t)c0 + 1 + kL2LChunk, nbox), wait_limit, withhold);
    }
}

// batched: chunk c of the queue is chunk c - off[s] of system s (chunks of
// kL2LChunk boxes from box 0, never across systems), so a box's parent is
// always earlier in the queue; every box first takes its unscaled M2L result
__global__ void __launch_bounds__(kWarpChildMax * 32)
k_b_l2l_down(const BatchSys *__restrict__ S, const int32_t *__restrict__ off, int nsys, int p,
             const double *__restrict__ gtab, const float2 *__restrict__ tab_df, unsigned long long *next,
             long long wait_limit, long long withhold) {
    extern __shared__ double2 sw[];
    const DF *tab = stage_child_tables_df(p, tab_df, sw);
    const int lane = threadIdx.x & 31;
    const int64_t total = off[nsys];
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(next, 1ull);
        c = __shfl_sync(0xffffffffu, c, 0);
        if ((int64_t)c >= total) break;
        const int s = batch_sys_of(off, nsys, (int64_t)c);
        const BatchSys &y = S[s];
        const TrIn a{y.centre, y.radius, (const BoxGeo *)y.box_geo, gtab, tab_df};
        const int64_t g0 = ((int64_t)c - off[s]) * kL2LChunk;
        l2l_chunk<true>(y.lw, p, a, y.Lh, y.L, tab, sw, y.done, y.err, g0,
                        std::min<int64_t>(g0 + kL2LChunk, y.nbox), wait_limit, withhold);
    }
}

}  // namespace

long double factl(int n) {
    long double r = 1.0L;
    for (int i = 2; i <= n; i++) r *= (long double)i;
    return r;
}

// Wigner d^n_{k m}(pi/2) by the explicit sum, in long double (the sum
// cancels; double loses ~5 digits by degree 20).
long double wigner_half_pi(int n, int k, int m) {
    long double tot = 0.0L;
    const long double c2n = powl(0.5L, (long double)n);
    for (int s = std::max(0, m - k); s <= std::min(n + m, n - k); s++) {
        const long double term =
            c2n / (factl(n + m - s) * factl(s) * factl(k - m + s) * factl(n - k - s));
        tot += ((k - m + s) & 1) ? -term : term;
    }
    return sqrtl(factl(n + k) * factl(n - k) * factl(n + m) * factl(n - m)) * tot;
}


// Tables for order p: D_n quadrants, axial coefficients, F_nm, 1/F_nm, 1/k.
std::vector<double> m2l_tables(int p) {
    std::vector<double> t;
    for (int n = 0; n <= p; n++)
        for (int k = 0; k <= n; k++)
            for (int m = 0; m <= n; m++) t.push_back((double)wigner_half_pi(n, k, m));
    auto F = [](int n, int m) { return sqrtl(factl(n + m) * factl(n - m)); };
    for (int l = 0; l <= p; l++)
        for (int k = l; k <= p; k++)
            for (int n = l; n <= p; n++) {
                long double a = factl(n + k) / (F(n, l) * F(k, l));
                t.push_back((double)(((k + l) & 1) ? -a : a));
            }
    for (int n = 0; n <= p; n++)
        for (int m = 0; m <= n; m++) t.push_back((double)F(n, m));
    for (int n = 0; n <= p; n++)
        for (int m = 0; m <= n; m++) t.push_back((double)(1.0L / F(n, m)));
    for (int k = 0; k <= p + 1; k++) t.push_back(k ? (double)(1.0L / k) : 0.0);  // 1/k
    return t;
}

PairTable pair_table(const Plan &P) {
    PairTable PT{};
    PT.lmin = 1;
    PT.lmax = std::max(P.B, 1);
    long long o = 0;
    for (int l = 0; l <= FMM_MAX_LEVELS + 1; l++) {
        if (l <= FMM_MAX_LEVELS && l >= 1 && l <= P.B) {
            PT.tgt[l] = P.wrow[l];
            PT.src[l] = P.wsrc[l];
        }
        PT.off[l] = o;
        if (l >= 1 && l <= P.B) o += P.nweak[l];
    }
    return PT;
}

int64_t total_weak(const Plan &P) {
    int64_t t = 0;
    for (int l = 1; l <= P.B; l++) t += P.nweak[l];
    return t;
}

cudaError_t allow_max_smem(const void *func, size_t need) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return e;
    const int room = optin - (int)fa.sharedSizeBytes;  // static shared memory counts against the limit
    if (need > (size_t)room) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, room);
}

// the tables of order p, computed once per process (long double sums of
// factorials: about a million operations at p = 12)
const std::vector<double> &m2l_tables_cached(int p) {
    static std::mutex mu;
    static std::vector<double> cache[FMM_MAX_P + 1];
    static bool ready[FMM_MAX_P + 1] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (!ready[p]) {
        cache[p] = m2l_tables(p);
        ready[p] = true;
    }
    return cache[p];
}

cudaError_t m2l_setup(Plan &P) {
    const std::vector<double> &t = m2l_tables_cached(P.p);
    P.m2l_ntab = (int)t.size();
    P.m2l_tab = (double *)palloc(P, t.size() * 8);
    P.m2m_arrive = (unsigned *)palloc(P, (size_t)P.nbox * 4);
    P.l2l_done = (int *)palloc(P, (size_t)P.nbox * 4);
    P.l2l_next = (unsigned long long *)palloc(P, 8);
    if (!P.m2l_tab || !P.m2m_arrive || !P.l2l_done || !P.l2l_next) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMemcpyAsync(P.m2l_tab, t.data(), t.size() * 8, cudaMemcpyHostToDevice, P.stream);
    if (e != cudaSuccess) return e;
    // stream-ordered copy from pageable memory completes before return
    if (P.prec == FMM_PREC_MIXED) {
        // double-float translations: the tables as (hi, lo) float pairs, and
        // the geometry of every box's translation to / from its parent
        std::vector<float2> tdf(t.size());
        for (size_t i = 0; i < t.size(); i++) {
            const float h = (float)t[i];
            tdf[i] = make_float2(h, (float)(t[i] - (double)h));
        }
        P.m2l_tab_df = (float2 *)palloc(P, tdf.size() * sizeof(float2));
        P.box_geo = palloc(P, (size_t)P.nbox * sizeof(BoxGeo));
        if (!P.m2l_tab_df || !P.box_geo) return cudaErrorMemoryAllocation;
        e = cudaMemcpyAsync(P.m2l_tab_df, tdf.data(), tdf.size() * sizeof(float2), cudaMemcpyHostToDevice, P.stream);
        if (e != cudaSuccess) return e;
        FMM_LAUNCH(k_box_geo, (unsigned)std::min<int64_t>((P.nbox + 255) / 256, (int64_t)sm_count() * 8), 256, 0,
                   P.stream, P.nbox, P.step, P.centre, P.radius, (BoxGeo *)P.box_geo);
    }
    const int nc = P.nc;
    int threads = 64;
    auto smem = [&](int T) { return (size_t)T * (nc + 2 * (P.p + 1)) * 16 + t.size() * 8; };
    if (smem(threads) > 220 * 1024) threads = 32;
    P.m2l_threads = threads;
    P.m2l_smem = smem(threads);
    e = allow_max_smem((const void *)k_m2l_rot_f64, P.m2l_smem);
    const size_t grp_max = (size_t)kWarpChildMax * warp_slice(P.p) * 16 + (size_t)warp_tabs(P.p) * 8;
    const void *kernels[] = {(const void *)k_l2l_warp<false>, (const void *)k_m2m_warp<false>,
                             (const void *)k_m2m_up<false>,   (const void *)k_l2l_down<false>,
                             (const void *)k_l2l_warp<true>,  (const void *)k_m2m_warp<true>,
                             (const void *)k_m2m_up<true>,    (const void *)k_l2l_down<true>};
    for (const void *k : kernels)
        if (e == cudaSuccess) e = allow_max_smem(k, grp_max);
    return e;
}

// M2M and L2L of the mixed form run in double-float arithmetic
static bool df_translations(const Plan &P) { return P.prec == FMM_PREC_MIXED && P.box_geo; }
static TrIn tr_in(const Plan &P) {
    return TrIn{P.centre, P.radius, (const BoxGeo *)P.box_geo, P.m2l_tab, P.m2l_tab_df};
}

// Warps (children) per block for a level of nch children: 8, or fewer so
// that the level still spreads over twice the SM count in blocks.
int warps_per_block(int64_t nch) {
    int w = kWarpChildMax;
    while (w > 1 && (nch + w - 1) / w < 2 * sm_count()) w >>= 1;
    return w;
}

size_t warp_child_smem(int p, int w) { return (size_t)w * warp_slice(p) * 16 + (size_t)warp_tabs(p) * 8; }

// parents of level l-step from their descendants at level l (parents zeroed first)
void m2m_level(Plan &P, int l) {
    const int64_t np = (int64_t)1 << (l - P.step), nch = (int64_t)1 << l;
    cudaMemsetAsync(P.M + (np - 1) * P.nc, 0, (size_t)np * P.nc * sizeof(double2), P.stream);
    const int w = warps_per_block(nch);
    if (df_translations(P))
        FMM_LAUNCH(k_m2m_warp<true>, (unsigned)((nch + w - 1) / w), 32 * w, warp_child_smem(P.p, w), P.stream, l,
                   P.step, P.p, tr_in(P), P.M);
    else
        FMM_LAUNCH(k_m2m_warp<false>, (unsigned)((nch + w - 1) / w), 32 * w, warp_child_smem(P.p, w), P.stream, l,
                   P.step, P.p, tr_in(P), P.M);
}

// level l from its ancestors at level l-step
void l2l_level(Plan &P, int l) {
    const int64_t nch = (int64_t)1 << l;
    const int w = warps_per_block(nch);
    if (df_translations(P))
        FMM_LAUNCH(k_l2l_warp<true>, (unsigned)((nch + w - 1) / w), 32 * w, warp_child_smem(P.p, w), P.stream, l,
                   P.step, P.p, tr_in(P), P.L);
    else
        FMM_LAUNCH(k_l2l_warp<false>, (unsigned)((nch + w - 1) / w), 32 * w, warp_child_smem(P.p, w), P.stream, l,
                   P.step, P.p, tr_in(P), P.L);
}

cudaError_t m2l_external(Plan &P, int level, int64_t n, const int32_t *tgt, const double2 *Msrc,
                         const double *csrc) {
    if (n == 0) return cudaGetLastError();
    PairTable PT{};
    PT.lmin = PT.lmax = level;
    PT.tgt[level] = tgt;
    PT.off[level] = 0;
    PT.off[level + 1] = n;
    FMM_LAUNCH(k_m2l_rot_f64, (unsigned)((n + P.m2l_threads - 1) / P.m2l_threads), P.m2l_threads, P.m2l_smem,
               P.stream, PT, P.p, P.centre, (const double2 *)nullptr, P.L_ext, P.m2l_tab, P.m2l_ntab, csrc, Msrc);
    return cudaGetLastError();
}

// Device-wide bounded waits of the one-launch downward pass: sleeps of
// ~0.1 us before the wait gives up, and a box whose flag is never raised
// (tests only; -1 = none). Set by fmm_set_wait_limit.
std::atomic<long long> g_wait_limit{1LL << 24};
std::atomic<long long> g_withhold{-1};

// the upward pass of binary levels in one launch, translations up to level `stop`
void m2m_up(Plan &P, int stop) {
    const int64_t nleaf = P.nleaf;
    cudaMemsetAsync(P.M, 0, (size_t)(nleaf - 1) * P.nc * sizeof(double2), P.stream);
    if (stop >= P.B) return;
    cudaMemsetAsync(P.m2m_arrive, 0, (size_t)P.nbox * 4, P.stream);
    const int w = kWarpChildMax;
    const unsigned grid = (unsigned)std::min<int64_t>((nleaf + w - 1) / w, (int64_t)sm_count() * 16);
    if (df_translations(P))
        FMM_LAUNCH(k_m2m_up<true>, grid, 32 * w, warp_child_smem(P.p, w), P.stream, P.B, stop, P.p, tr_in(P), P.M,
                   P.m2m_arrive);
    else
        FMM_LAUNCH(k_m2m_up<false>, grid, 32 * w, warp_child_smem(P.p, w), P.stream, P.B, stop, P.p, tr_in(P), P.M,
                   P.m2m_arrive);
}

// the downward pass of binary levels in one launch; boxes whose parent level
// is below lw receive nothing
void l2l_down(Plan &P, int lw) {
    if (P.B == 0) return;
    cudaMemsetAsync(P.l2l_done, 0, (size_t)P.nbox * 4, P.stream);
    cudaMemsetAsync(P.l2l_next, 0, 8, P.stream);
    const int w = kWarpChildMax;
    const int64_t items = (P.nbox + kL2LChunk - 1) / kL2LChunk;
    const unsigned grid = (unsigned)std::min<int64_t>((items + w - 1) / w, (int64_t)sm_count() * 8);
    if (df_translations(P))
        FMM_LAUNCH(k_l2l_down<true>, grid, 32 * w, warp_child_smem(P.p, w), P.stream, P.B, lw, P.p, tr_in(P), P.L,
                   P.l2l_done, P.l2l_next, P.d_err, g_wait_limit.load(), g_withhold.load());
    else
        FMM_LAUNCH(k_l2l_down<false>, grid, 32 * w, warp_child_smem(P.p, w), P.stream, P.B, lw, P.p, tr_in(P), P.L,
                   P.l2l_done, P.l2l_next, P.d_err, g_wait_limit.load(), g_withhold.load());
}

// FP64 M2L over all levels in one launch; accumulates into L (zeroed first)
cudaError_t m2l_all(Plan &P) {
    cudaMemsetAsync(P.L, 0, (size_t)P.nbox * P.nc * sizeof(double2), P.stream);
    const int64_t tot = total_weak(P);
    if (tot == 0) return cudaGetLastError();
    FMM_LAUNCH(k_m2l_rot_f64, (unsigned)((tot + P.m2l_threads - 1) / P.m2l_threads), P.m2l_threads,
               P.m2l_smem, P.stream, pair_table(P), P.p, P.centre, P.M, P.L, P.m2l_tab, P.m2l_ntab);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Single-precision rotational M2L (FMM_PREC_MIXED).
//
// Same five steps, on scaled coefficients: the source multipole is read as
// Mhat_n = M_n / r_s^n (float, prepared once per box) and the contribution is
// formed as Lhat_k = r_t^k L_k, so the translation becomes
//   Lhat r_k^l = (1/rho) (r_t/rho)^k sum_n A(k,n,l) (r_s/rho)^n conj(Mhat r_n^l)
// with r_s/rho, r_t/rho < 1 for every weak pair: all float values stay O(1).
// The target's local expansion is accumulated in double.
//
// GPU mapping: one weak pair per thread, all levels in one launch (pairs
// sorted by target), blocks striding over chunks of 128 pairs. Every degree
// (and every two orders of the translation) is its own template instance,
// so a degree's input vector sits in registers; a fold's outputs come from a
// runtime loop, two per iteration (one of each parity), each a dot product
// of packed pairs -- (Re of one parity, Im of the other) against a row of
// matching coefficient pairs -- in FFMA2. The coefficient rows are staged in
// shared memory once per block and read at warp-uniform addresses, so the
// code stays a few thousand instructions that loop instead of a straight
// line of every multiply-add. Between the stages the pair's coefficients sit
// in its lane of tensor memory (degrees 0..9) and in a shared-memory column
// (higher degrees); outputs that feed another fold are stored in the pair
// layout that fold reads.
// ---------------------------------------------------------------------------
namespace {


// Packed coefficient-pair tables of order P (float4 = two pairs), built per
// plan and staged in shared memory. A fold table has, per degree n and
// output k = 0..n, jp(n) float4 holding the pairs (G_{k,2j}, G_{k,2j+1}) when
// n+k is even and (G_{k,2j+1}, G_{k,2j}) when odd, zero past column n, for
//   Df   (forward, first fold)   G_km = D_km F_nm (m?2:1) (k?2:1)
//   DTf  (forward, second fold)  G_km = D_mk
//   Db   (inverse, first fold)   G_km = D_km (m?2:1) (k?2:1)
//   DTb  (inverse, second fold)  G_km = D_mk F_nk
// (D = d^n(pi/2); the real factors of the rotation are folded in), at
// offsets 0, 1, 2, 3 times dpo(P+1); then the axial rows: order l, output
// k = l..P, ja(P,l) float4 of (A(k,n,l), A(k,n,l)) for n = l..P, zero-padded.
// The i^m of the forward rotation and the i^-m of the inverse one cancel
// through the conjugate of the translation, so neither is applied.
__host__ __device__ constexpr int jp_of(int n) { return (n + 4) / 4; }
__host__ __device__ constexpr int dpo(int n) { return n <= 0 ? 0 : dpo(n - 1) + n * jp_of(n - 1); }
__host__ __device__ constexpr int ja_of(int P, int l) { return (P + 2 - l) / 2; }
__host__ __device__ constexpr int apo(int P, int l) {
    return l <= 0 ? 0 : apo(P, l - 1) + (P + 2 - l) * ja_of(P, l - 1);
}
__host__ __device__ constexpr int pair_tab_len(int P) { return 4 * dpo(P + 1) + apo(P, P + 1); }

__device__ __forceinline__ float2 fmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// Per-pair coefficient storage between the stages: degrees 0..kTmDeg live
// in the thread's lane of tensor memory (Re, Im interleaved: columns
// 2 tri(n,m), 2 tri(n,m)+1), the rest in a shared-memory column of the
// block (stride T). Tensor memory is otherwise idle in this kernel; moving
// 55 of the 91 coefficients (p = 12) there cuts shared memory per block from
// 111 to 55 KB, so three blocks (12 warps, register-limited) fit an SM
// instead of two.
constexpr int kTmDeg = 9;
constexpr int kTmC = (kTmDeg + 1) * (kTmDeg + 2) / 2;  // first coefficient in shared memory

struct VS {
    float2 *s;    // shared column of this thread: coefficient c at s[(c - kTmC) * T]
    uint32_t t;   // this thread's tensor-memory lane, column 0
    int T;
    uint32_t ph;  // this thread's lane of the phase columns: e^{ik beta} at 2k, 2k+1
};

template <int X>
__device__ __forceinline__ void tm_st(uint32_t a, const float *v) {
    if constexpr (X == 1)
        asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(a), "f"(v[0]));
    else if constexpr (X == 2)
        asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};" ::"r"(a), "f"(v[0]), "f"(v[1]));
    else if constexpr (X == 4)
        asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(a), "f"(v[0]),
                     "f"(v[1]), "f"(v[2]), "f"(v[3]));
    else if constexpr (X == 8)
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(a),
                     "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]));
    else
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
            "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(a),
            "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]),
            "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]));
}

template <int X>
__device__ __forceinline__ void tm_ld(uint32_t a, float *v) {
    if constexpr (X == 1)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=f"(v[0]) : "r"(a));
    else if constexpr (X == 2)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=f"(v[0]), "=f"(v[1]) : "r"(a));
    else if constexpr (X == 4)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                     : "r"(a));
    else if constexpr (X == 8)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
                       "=f"(v[7])
                     : "r"(a));
    else
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]),
              "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]),
              "=f"(v[15])
            : "r"(a));
}

// columns [OFF, OFF + REM) in power-of-two chunks
template <int OFF, int REM>
struct TCols {
    static __device__ __forceinline__ void st(uint32_t a, const float *v) {
        constexpr int X = REM >= 16 ? 16 : REM >= 8 ? 8 : REM >= 4 ? 4 : REM >= 2 ? 2 : 1;
        if constexpr (REM > 0) {
            tm_st<X>(a + OFF, v + OFF);
            TCols<OFF + X, REM - X>::st(a, v);
        }
    }
    static __device__ __forceinline__ void ld(uint32_t a, float *v) {
        constexpr int X = REM >= 16 ? 16 : REM >= 8 ? 8 : REM >= 4 ? 4 : REM >= 2 ? 2 : 1;
        if constexpr (REM > 0) {
            tm_ld<X>(a + OFF, v + OFF);
            TCols<OFF + X, REM - X>::ld(a, v);
        }
    }
};

__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// the loaded registers are valid only after the wait: the empty asm ties
// every later use of them to a point after it
template <int K>
__device__ __forceinline__ void tm_wait_ld(float *v) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < K; j++) asm volatile("" : "+f"(v[j]));
}

template <int N>
__device__ __forceinline__ void v_get_deg(const VS &vs, float2 (&u)[N + 1]) {
    if constexpr (N <= kTmDeg) {
        float f[2 * (N + 1)];
        TCols<0, 2 * (N + 1)>::ld(vs.t + 2 * tri(N, 0), f);
        tm_wait_ld<2 * (N + 1)>(f);
#pragma unroll
        for (int m = 0; m <= N; m++) u[m] = make_float2(f[2 * m], f[2 * m + 1]);
    } else {
#pragma unroll
        for (int m = 0; m <= N; m++) u[m] = vs.s[(tri(N, m) - kTmC) * vs.T];
    }
}

// coefficient c of degree N of the pair's storage (where it lives is fixed by N)
template <int N>
__device__ __forceinline__ void v_put_deg(const VS &vs, int c, float2 v) {
    if constexpr (N <= kTmDeg) {
        const float f[2] = {v.x, v.y};
        tm_st<2>(vs.t + 2 * c, f);
    } else {
        vs.s[(c - kTmC) * vs.T] = v;
    }
}

// coefficient c (run time) of the pair's storage
__device__ __forceinline__ void v_put_rt(const VS &vs, int c, float2 v) {
    if (c < kTmC) {  // warp-uniform
        const float f[2] = {v.x, v.y};
        tm_st<2>(vs.t + 2 * c, f);
    } else {
        vs.s[(c - kTmC) * vs.T] = v;
    }
}

// (Re v_{2j}, Im v_{2j+1}) and (Re v_{2j+1}, Im v_{2j}), zero past m = N
template <int N>
struct Pairs {
    float2 e[2 * jp_of(N)], o[2 * jp_of(N)];
};

template <int N>
__device__ __forceinline__ void make_pairs(const float2 (&v)[N + 1], Pairs<N> &q) {
#pragma unroll
    for (int j = 0; j < 2 * jp_of(N); j++) {
        const float2 a = 2 * j <= N ? v[2 * j] : make_float2(0.f, 0.f);
        const float2 b = 2 * j + 1 <= N ? v[2 * j + 1] : make_float2(0.f, 0.f);
        q.e[j] = make_float2(a.x, b.y);
        q.o[j] = make_float2(b.x, a.y);
    }
}

// The first fold's outputs x_k, x_{k+1} (k even) go to the degree's slots k,
// k+1 as (Re x_k, Im x_{k+1}) and (Re x_{k+1}, Im x_k): read back, they are
// the pair operands of the second fold as they stand. A last unpaired output
// (N even) keeps (Re x_N, Im x_N).
template <int N>
__device__ __forceinline__ void put_paired(const VS &vs, int c, float2 a0, float2 a1) {
    if constexpr (N <= kTmDeg) {
        const float f[4] = {a0.x, a1.y, a1.x, a0.y};
        tm_st<4>(vs.t + 2 * c, f);
    } else {
        vs.s[(c - kTmC) * vs.T] = make_float2(a0.x, a1.y);
        vs.s[(c + 1 - kTmC) * vs.T] = make_float2(a1.x, a0.y);
    }
}

// the pair operands of degree N from slots written by put_paired
template <int N>
__device__ __forceinline__ void get_paired(const VS &vs, Pairs<N> &q) {
    float2 u[N + 1];
    v_get_deg<N>(vs, u);
#pragma unroll
    for (int j = 0; j < 2 * jp_of(N); j++) {
        if (2 * j + 1 <= N) {
            q.e[j] = u[2 * j];
            q.o[j] = u[2 * j + 1];
        } else if (2 * j == N) {
            q.e[j] = make_float2(u[N].x, 0.f);
            q.o[j] = make_float2(0.f, u[N].y);
        } else {
            q.e[j] = q.o[j] = make_float2(0.f, 0.f);
        }
    }
}

// sum_j row_j * w_j over J float4 (two pairs each), two packed accumulators
template <int J>
__device__ __forceinline__ float2 dot_row(const float4 *__restrict__ row, const float2 *w) {
    float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < J; q++) {
        const float4 d = row[q];
        a0 = __ffma2_rn(make_float2(d.x, d.y), w[2 * q], a0);
        a1 = __ffma2_rn(make_float2(d.z, d.w), w[2 * q + 1], a1);
    }
    return __fadd2_rn(a0, a1);
}

// out2(k, fold_k, fold_k+1) for even k < N and out1(N, fold_N) when N is
// even, over the rows of degree N; the output's parity (N + k) picks the pair set
template <int N, typename Out2, typename Out1>
__device__ __forceinline__ void fold_rt2(const float4 *__restrict__ rows, const Pairs<N> &q, Out2 &&out2,
                                         Out1 &&out1) {
    constexpr int J = jp_of(N);
    const float2 *w0 = (N & 1) ? q.o : q.e;
    const float2 *w1 = (N & 1) ? q.e : q.o;
#pragma unroll 1
    for (int k = 0; k < N; k += 2) {
        const float2 a0 = dot_row<J>(rows + k * J, w0);
        const float2 a1 = dot_row<J>(rows + (k + 1) * J, w1);
        out2(k, a0, a1);
    }
    if constexpr ((N & 1) == 0) out1(N, dot_row<J>(rows + N * J, w0));
}

// The first fold of either rotation multiplies output k by e^{ik beta}
// (doubled for k > 0 in the tables): the powers are formed once per pair into
// tensor-memory columns, and each iteration reads its two with one load
// issued before the iteration's products.
template <int N, typename Put2, typename Put1>
__device__ __forceinline__ void fold1_phased(const float4 *__restrict__ rows, const Pairs<N> &q, const VS &vs,
                                             Put2 &&put2, Put1 &&put1) {
    constexpr int J = jp_of(N);
    const float2 *w0 = (N & 1) ? q.o : q.e;
    const float2 *w1 = (N & 1) ? q.e : q.o;
#pragma unroll 1
    for (int k = 0; k < N; k += 2) {
        float f[4];
        tm_ld<4>(vs.ph + 2 * k, f);
        const float2 a0 = dot_row<J>(rows + k * J, w0);
        const float2 a1 = dot_row<J>(rows + (k + 1) * J, w1);
        tm_wait_ld<4>(f);
        put2(k, fmulc(a0, make_float2(f[0], f[1])), fmulc(a1, make_float2(f[2], f[3])));
    }
    if constexpr ((N & 1) == 0) {
        float f[2];
        tm_ld<2>(vs.ph + 2 * N, f);
        const float2 a = dot_row<J>(rows + N * J, w0);
        tm_wait_ld<2>(f);
        put1(N, fmulc(a, make_float2(f[0], f[1])));
    }
}

// out(k, fold_k) for k = 0..N of the fold with the rows of degree N
template <int N, typename Out>
__device__ __forceinline__ void fold_rt(const float4 *__restrict__ rows, const Pairs<N> &q, Out &&out) {
    fold_rt2<N>(rows, q, [&](int k, float2 a0, float2 a1) {
        out(k, a0);
        out(k + 1, a1);
    }, out);
}

// forward rotation of degree N of the scaled source multipole into the
// storage
template <int P, int N>
__device__ __forceinline__ void fwd_deg(const float2 *__restrict__ Ms, const VS &vs, bool valid, float2 eai,
                                        const float4 *__restrict__ tab) {
    // the degree's coefficients, two per 16-byte load where the pair is aligned
    constexpr int c0 = N * (N + 1) / 2, m0 = c0 & 1;
    float2 u[N + 1];
#pragma unroll
    for (int m = 0; m <= N; m++) u[m] = make_float2(0.f, 0.f);
    if (valid) {
        if constexpr (m0 == 1) u[0] = Ms[c0];
#pragma unroll
        for (int m = m0; m + 1 <= N; m += 2) {
            const float4 t = *(const float4 *)(Ms + c0 + m);
            u[m] = make_float2(t.x, t.y);
            u[m + 1] = make_float2(t.z, t.w);
        }
        if constexpr (((N + 1 - m0) & 1) == 1) u[N] = Ms[c0 + N];
    }
    float2 ph = make_float2(1.f, 0.f);
#pragma unroll
    for (int m = 0; m <= N; m++) {
        u[m] = fmulc(u[m], ph);
        ph = fmulc(ph, eai);
    }
    Pairs<N> q;
    make_pairs<N>(u, q);
    // the first fold's outputs go through the degree's own (still empty) slots
    fold1_phased<N>(tab + dpo(N), q, vs, [&](int k, float2 x0, float2 x1) { put_paired<N>(vs, c0 + k, x0, x1); },
                    [&](int k, float2 x) { v_put_deg<N>(vs, c0 + k, x); });
    if constexpr (N <= kTmDeg) tm_wait_st();
    get_paired<N>(vs, q);
    fold_rt<N>(tab + dpo(P + 1) + dpo(N), q, [&](int m, float2 a) { v_put_deg<N>(vs, c0 + m, a); });
    if constexpr (N <= kTmDeg) tm_wait_st();
}

// Floats of a warp's transpose buffer: column-major with a column stride of
// 36 floats (lane i of column c at 36 c + i: conflict-free writes, 16-byte
// column reads).
constexpr int kRedCol = 36;
template <int P>
__host__ __device__ constexpr int region_floats() { return 2 * (P + 1) * kRedCol; }

// Segmented sum of one contribution over runs of equal target (warp-wide:
// every lane calls it) and the add of each run's sum into its target's
// coefficient; out of line, as warps with mixed targets are the rare case.
__device__ __noinline__ void seg_add(float sx, float sy, unsigned same_mask, bool head, double2 *dst) {
#pragma unroll
    for (int j = 0; j < 5; j++) {
        const float ox = __shfl_down_sync(0xffffffffu, sx, 1 << j);
        const float oy = __shfl_down_sync(0xffffffffu, sy, 1 << j);
        if ((same_mask >> j) & 1u) {
            sx += ox;
            sy += oy;
        }
    }
    if (head) {
        atomicAdd(&dst->x, (double)sx);
        atomicAdd(&dst->y, (double)sy);
    }
}

// Column sums of a warp's transpose buffer (2 (N+1) columns: Re of orders
// 0..N, then Im) into the target's coefficients c0..c0+N.
__device__ __forceinline__ void col_add(const float *red, int N, double2 *dst) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    for (int col = lane; col < 2 * (N + 1); col += 32) {
        const float4 *c4 = (const float4 *)(red + col * kRedCol);
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const float4 v = c4[i];
            a0 = __fadd2_rn(a0, make_float2(v.x, v.y));
            a1 = __fadd2_rn(a1, make_float2(v.z, v.w));
        }
        const float s = (a0.x + a0.y) + (a1.x + a1.y);
        const int l = col <= N ? col : col - (N + 1);
        atomicAdd((double *)&dst[l] + (col <= N ? 0 : 1), (double)s);
    }
}

// inverse rotation of degree N, then the sum over the warp's pairs into the
// scaled local Lh (double) of their target: a warp whose valid lanes share
// one target (the common case: the pair list is sorted by target) transposes
// its 2 (N+1) values per lane through shared memory and adds each column with
// one atomic; otherwise a segmented shuffle sum over runs of equal target
template <int P, int N>
__device__ __forceinline__ void bwd_deg(const VS &vs, float2 eai, double2 *__restrict__ Lh,
                                        unsigned same_mask, bool head, int uniform_tgt,
                                        double2 *__restrict__ Lbase, const float4 *__restrict__ tab, float *red) {
    constexpr int NC = (P + 1) * (P + 2) / 2, DP = dpo(P + 1);
    Pairs<N> q;
    get_paired<N>(vs, q);  // the translation left the degree in the pair layout
    // the first fold's outputs go through the degree's slots (read above)
    fold1_phased<N>(tab + 2 * DP + dpo(N), q, vs,
                    [&](int j, float2 x0, float2 x1) { put_paired<N>(vs, tri(N, 0) + j, x0, x1); },
                    [&](int j, float2 x) { v_put_deg<N>(vs, tri(N, 0) + j, x); });
    if constexpr (N <= kTmDeg) tm_wait_st();
    get_paired<N>(vs, q);
    const int lane = threadIdx.x & 31;
    const bool uni = uniform_tgt >= 0;  // warp-uniform
    float2 ph = make_float2(1.f, 0.f);
    fold_rt<N>(tab + 3 * DP + dpo(N), q, [&](int l, float2 a) {
        const float2 t = fmulc(a, ph);  // (-i e^{ia})^l
        ph = fmulc(ph, eai);
        const float rx = t.x, ry = t.y;
        if (uni) {
            red[l * kRedCol + lane] = rx;
            red[(N + 1 + l) * kRedCol + lane] = ry;
        } else {
            seg_add(rx, ry, same_mask, head, &Lh[tri(N, 0) + l]);
        }
    });
    if (uni) col_add(red, N, Lbase + (int64_t)uniform_tgt * NC + tri(N, 0));
    __syncwarp();  // the next degree reuses the region
}

// column L (degrees n = L..P) of the storage, conjugated and scaled by qs^n,
// as the packed operands of the translation rows (zero past P)
template <int P, int L, int J>
__device__ __forceinline__ void axial_col(const VS &vs, float qs, float2 (&s)[2 * J]) {
    constexpr int len = P + 1 - L;
    constexpr int ntm = L > kTmDeg ? 0 : (P < kTmDeg ? P : kTmDeg) + 1 - L;  // of them in tensor memory
    float f[2 * len];
#pragma unroll
    for (int n = L; n <= P; n++) {
        if (n <= kTmDeg) {
            tm_ld<2>(vs.t + 2 * tri(n, L), f + 2 * (n - L));
        } else {
            const float2 v = vs.s[(tri(n, L) - kTmC) * vs.T];
            f[2 * (n - L)] = v.x;
            f[2 * (n - L) + 1] = v.y;
        }
    }
    if constexpr (ntm > 0) tm_wait_ld<2 * ntm>(f);
    float sp = 1.f;
#pragma unroll
    for (int j = 0; j < L; j++) sp *= qs;
#pragma unroll
    for (int n = 0; n < 2 * J; n++) {
        s[n] = n < len ? make_float2(f[2 * n] * sp, -f[2 * n + 1] * sp) : make_float2(0.f, 0.f);
        sp *= qs;
    }
}

// translation along z of orders L and L+1 (L even), in place in the storage;
// qs = r_s / rho, qt = r_t / rho. The outputs of degree k go to slots L, L+1
// as (Re of order L, Im of order L+1) and (Re of L+1, Im of L), the pair
// layout the inverse rotation's first fold reads; order L alone at k = L (the
// last slot of an even degree) keeps (Re, Im).
template <int P, int L>
__device__ __forceinline__ void axial_ord(const VS &vs, float qs, float qt, float rinv,
                                          const float4 *__restrict__ tab) {
    constexpr int J0 = ja_of(P, L), J1 = ja_of(P, L + 1);
    float2 s0[2 * J0];
    axial_col<P, L, J0>(vs, qs, s0);
    float tp = rinv;
#pragma unroll
    for (int j = 0; j < L; j++) tp *= qt;
    const float4 *rows0 = tab + 4 * dpo(P + 1) + apo(P, L);
    {
        const float2 a = dot_row<J0>(rows0, s0);
        v_put_rt(vs, tri(L, L), make_float2(a.x * tp, a.y * tp));
        tp *= qt;
    }
    if constexpr (L + 1 <= P) {
        float2 s1[2 * J1];
        axial_col<P, L + 1, J1>(vs, qs, s1);
        const float4 *rows1 = tab + 4 * dpo(P + 1) + apo(P, L + 1);
#pragma unroll 1
        for (int k = L + 1; k <= P; k++) {
            const float2 a0 = dot_row<J0>(rows0 + (k - L) * J0, s0);
            const float2 a1 = dot_row<J1>(rows1 + (k - L - 1) * J1, s1);
            const int c = tri(k, L);
            const float2 x0 = make_float2(a0.x * tp, a0.y * tp), x1 = make_float2(a1.x * tp, a1.y * tp);
            if (k <= kTmDeg) {  // warp-uniform
                const float f[4] = {x0.x, x1.y, x1.x, x0.y};
                tm_st<4>(vs.t + 2 * c, f);
            } else {
                vs.s[(c - kTmC) * vs.T] = make_float2(x0.x, x1.y);
                vs.s[(c + 1 - kTmC) * vs.T] = make_float2(x1.x, x0.y);
            }
            tp *= qt;
        }
    }
    if constexpr (L <= kTmDeg) tm_wait_st();
}

template <int P, int N>
struct Seq {
    __device__ static __forceinline__ void fwd(const float2 *Ms, const VS &vs, bool valid, float2 eai,
                                               const float4 *tab) {
        fwd_deg<P, N>(Ms, vs, valid, eai, tab);
        Seq<P, N + 1>::fwd(Ms, vs, valid, eai, tab);
    }
    __device__ static __forceinline__ void axial(const VS &vs, float qs, float qt, float rinv, const float4 *tab) {
        if constexpr ((N & 1) == 0) axial_ord<P, N>(vs, qs, qt, rinv, tab);
        Seq<P, N + 1>::axial(vs, qs, qt, rinv, tab);
    }
    __device__ static __forceinline__ void bwd(const VS &vs, float2 eai, double2 *Lh, unsigned same,
                                               bool head, int ut, double2 *Lbase, const float4 *tab, float *red) {
        bwd_deg<P, N>(vs, eai, Lh, same, head, ut, Lbase, tab, red);
        Seq<P, N + 1>::bwd(vs, eai, Lh, same, head, ut, Lbase, tab, red);
    }
};
template <int P>
struct Seq<P, P + 1> {
    __device__ static __forceinline__ void fwd(const float2 *, const VS &, bool, float2, const float4 *) {}
    __device__ static __forceinline__ void axial(const VS &, float, float, float, const float4 *) {}
    __device__ static __forceinline__ void bwd(const VS &, float2, double2 *, unsigned, bool, int, double2 *,
                                               const float4 *, float *) {}
};

constexpr int kF32Threads = 128;

// coefficients of order P kept in tensor memory / in shared memory, and the
// tensor-memory columns a block allocates (a power of two, at least 32)
template <int P>
struct VSplit {
    static constexpr int NC = (P + 1) * (P + 2) / 2;
    static constexpr int NT = NC < kTmC ? NC : kTmC;
    static constexpr int NS = NC - NT;
    static constexpr int COLS = 2 * NT <= 32 ? 32 : 2 * NT <= 64 ? 64 : 128;
    static constexpr int PHC = 2 * (P + 1) <= 32 ? 32 : 64;  // columns of the e^{ik beta} table
    // shared bytes: the storage columns, per warp the transpose
    // region, then the coefficient-pair tables
    static constexpr size_t TAB = (size_t)kF32Threads * NS * 8 + (size_t)(kF32Threads / 32) * region_floats<P>() * 4;
    static constexpr size_t SMEM = TAB + (size_t)pair_tab_len(P) * 16;
};

// one chunk of 128 pairs (pair g for this thread; lanes past the end carry zeros)
template <int P>
__device__ __forceinline__ void m2l_chunk(const PairTable &PT, const float4 *__restrict__ cf,
                                          const float2 *__restrict__ Mf,
                                          double2 *__restrict__ Lh, const float4 *tab, int64_t g, int64_t npairs,
                                          float2 *smf, uint32_t tbase, uint32_t tphase) {
    using SP = VSplit<P>;
    constexpr int NC = SP::NC;
    const int tid = threadIdx.x, warp = tid >> 5;
    const bool valid = g < npairs;
    int64_t gt = -1, gs = 0;
    float dx = 1.f, dy = 0.f, dz = 0.f, rs = 1.f, rt = 1.f;
    if (valid) {
        pair_of(PT, g, gt, gs);
        // the centre offset from the split centres: the hi difference and its
        // rounding error (TwoSum), plus the lo difference, rounded once: the
        // double difference rounded to float, without double arithmetic
        const float4 th = cf[2 * gt], tl = cf[2 * gt + 1], sh = cf[2 * gs], sl = cf[2 * gs + 1];
        dx = offset_f(th.x, sh.x, tl.x, sl.x);
        dy = offset_f(th.y, sh.y, tl.y, sl.y);
        dz = offset_f(th.z, sh.z, tl.z, sl.z);
        rs = sh.w > 0.f ? sh.w : 1.f;
        rt = th.w > 0.f ? th.w : 1.f;
    }
    bool same[5], head;
    seg_setup(gt, same, head);
    unsigned same_mask = 0;
#pragma unroll
    for (int j = 0; j < 5; j++) same_mask |= (unsigned)same[j] << j;
    const float rxy2 = fmaf(dx, dx, dy * dy);
    const float rxy = sqrtf(rxy2), rinv = rsqrtf(fmaf(dz, dz, rxy2));
    const float rxinv = rxy > 0.f ? 1.f / rxy : 0.f;
    const float2 ea = rxy > 0.f ? make_float2(dx * rxinv, dy * rxinv) : make_float2(1.f, 0.f);
    const float2 ebv = make_float2(dz * rinv, rxy * rinv);
    const float2 eai = make_float2(ea.y, -ea.x);
    const float qs = rs * rinv, qt = rt * rinv;
    // every lane runs every stage (tensor-memory accesses are warp-wide); a
    // lane without a pair carries zeros
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
    const VS vs{smf + tid, tbase + lanes, kF32Threads, tphase + lanes};
    {
        float f[2 * (P + 1)];
        float2 pb = make_float2(1.f, 0.f);
#pragma unroll
        for (int k = 0; k <= P; k++) {
            f[2 * k] = pb.x;
            f[2 * k + 1] = pb.y;
            pb = fmulc(pb, ebv);
        }
        TCols<0, 2 * (P + 1)>::st(vs.ph, f);
        tm_wait_st();
    }
    float *region = (float *)(smf + SP::NS * kF32Threads) + warp * region_floats<P>();
    Seq<P, 0>::fwd(Mf + gs * mf_stride(P), vs, valid, eai, tab);
    Seq<P, 0>::axial(vs, qs, qt, rinv, tab);
    // the warp's pairs share one target (invalid lanes add zeros): transpose path
    const int t32 = gt >= 0 ? (int)gt : -1;
    const int tmax = __reduce_max_sync(0xffffffffu, t32);
    const bool uniform = __all_sync(0xffffffffu, t32 == tmax || t32 < 0);
    Seq<P, 0>::bwd(vs, eai, Lh + (gt >= 0 ? gt : 0) * NC, same_mask, head, uniform ? tmax : -1, Lh, tab, region);
}

// one weak pair per thread, all levels, blocks striding over chunks of 128
// pairs; accumulates r_t^k L_k into Lh
template <int P>
__global__ void __launch_bounds__(kF32Threads, 3)
k_m2l_rot_f32(PairTable PT, const float4 *__restrict__ cf, const float2 *__restrict__ Mf,
              double2 *__restrict__ Lh, const float4 *__restrict__ gtab) {
    using SP = VSplit<P>;
    extern __shared__ float2 smf[];  // [NS][threads], the per-warp regions, the tables
    __shared__ uint32_t s_tmem, s_tphase;
    const int tid = threadIdx.x, warp = tid >> 5;
    float4 *tab = (float4 *)((char *)smf + SP::TAB);
    for (int i = tid; i < pair_tab_len(P); i += kF32Threads) tab[i] = gtab[i];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&s_tmem)),
                     "r"(SP::COLS));
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&s_tphase)),
                     "r"(SP::PHC));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = s_tmem, tphase = s_tphase;
    const int64_t npairs = PT.off[PT.lmax + 1];
    for (int64_t g0 = blockIdx.x * (int64_t)kF32Threads; g0 < npairs; g0 += (int64_t)gridDim.x * kF32Threads)
        m2l_chunk<P>(PT, cf, Mf, Lh, tab, g0 + tid, npairs, smf, tbase, tphase);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(SP::COLS));
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tphase), "r"(SP::PHC));
    }
}

// batched: the 128-pair chunks of every system of the same order in one launch
template <int P>
__global__ void __launch_bounds__(kF32Threads, 3)
k_b_m2l_rot_f32(const BatchSys *__restrict__ S, const int32_t *__restrict__ off, int nsys,
                const float4 *__restrict__ gtab) {
    using SP = VSplit<P>;
    extern __shared__ float2 smf[];  // [NS][threads], the per-warp regions, the tables
    __shared__ uint32_t s_tmem, s_tphase;
    const int tid = threadIdx.x, warp = tid >> 5;
    float4 *tab = (float4 *)((char *)smf + SP::TAB);
    for (int i = tid; i < pair_tab_len(P); i += kF32Threads) tab[i] = gtab[i];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&s_tmem)),
                     "r"(SP::COLS));
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&s_tphase)),
                     "r"(SP::PHC));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = s_tmem, tphase = s_tphase;
    // chunk c of the batch is chunk c - off[s] of system s (128 pairs each)
    const int64_t nchunks = off[nsys];
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int s = batch_sys_of(off, nsys, c);
        const BatchSys &y = S[s];
        m2l_chunk<P>(y.pt, y.box_cf, y.Mf, y.Lh, tab, (c - off[s]) * kF32Threads + tid, y.npairs, smf,
                     tbase, tphase);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(SP::COLS));
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tphase), "r"(SP::PHC));
    }
}

// Mhat = M / r^n in float, every box (levels >= 1)
__global__ void k_scale_multipoles(int64_t nbox, int p, const double *__restrict__ radius,
                                   const double2 *__restrict__ M, float2 *__restrict__ Mf) {
    const int nc = ncoef(p), lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < nbox; g += nw) {
        const double pw = inv_radius_pow(radius, g, p, lane);
        for (int c0 = 0; c0 < nc; c0 += 32) {  // warp-uniform trip count around the shuffle
            const int c = c0 + lane;
            const double s = __shfl_sync(0xffffffffu, pw, degree_of(min(c, nc - 1)));
            if (c < nc) {
                const double2 m = M[g * nc + c];
                Mf[g * mf_stride(p) + c] = make_float2((float)(m.x * s), (float)(m.y * s));
            }
        }
    }
}

// L = Lhat / r^n, every box
__global__ void k_unscale_locals(int64_t nbox, int p, const double *__restrict__ radius,
                                 const double2 *__restrict__ Lh, double2 *__restrict__ L) {
    const int nc = ncoef(p), lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < nbox; g += nw) {
        const double pw = inv_radius_pow(radius, g, p, lane);
        for (int c0 = 0; c0 < nc; c0 += 32) {
            const int c = c0 + lane;
            const double s = __shfl_sync(0xffffffffu, pw, degree_of(min(c, nc - 1)));
            if (c < nc) {
                const double2 h = Lh[g * nc + c];
                L[g * nc + c] = make_double2(h.x * s, h.y * s);
            }
        }
    }
}

long double norm_F(int n, int m) { return sqrtl(factl(n + m) * factl(n - m)); }

// entry (k, m) of fold table `tab` (Df, DTf, Db, DTb) of degree n, zero past m = n
float fold_entry(int tab, int n, int k, int m) {
    if (m > n) return 0.f;
    const bool tr = tab & 1;
    long double g = tr ? wigner_half_pi(n, m, k) : wigner_half_pi(n, k, m);
    if (!tr) g *= (m ? 2.0L : 1.0L) * (k ? 2.0L : 1.0L);
    if (tab == 0) g *= norm_F(n, m);
    if (tab == 3) g *= norm_F(n, k);
    return (float)g;
}

// entry (k, n) of the translation table of order l, zero past n = p
float axial_entry(int p, int l, int k, int n) {
    if (n > p) return 0.f;
    const long double a = factl(n + k) / (norm_F(n, l) * norm_F(k, l));
    return (float)(((k + l) & 1) ? -a : a);
}

// the packed pair tables of order p (layout at jp_of / dpo / ja_of / apo)
std::vector<float4> f32_pair_tables(int p) {
    std::vector<float4> t;
    t.reserve(pair_tab_len(p));
    for (int tab = 0; tab < 4; tab++)  // Df, DTf, Db, DTb
        for (int n = 0; n <= p; n++)
            for (int k = 0; k <= n; k++) {
                auto G = [&](int m) { return fold_entry(tab, n, k, m); };
                const bool odd = (n + k) & 1;
                for (int q = 0; q < jp_of(n); q++) {
                    const int a = 4 * q;  // pairs 2q, 2q+1 cover m = a .. a+3
                    t.push_back(odd ? make_float4(G(a + 1), G(a), G(a + 3), G(a + 2))
                                    : make_float4(G(a), G(a + 1), G(a + 2), G(a + 3)));
                }
            }
    for (int l = 0; l <= p; l++)
        for (int k = l; k <= p; k++) {
            for (int q = 0; q < ja_of(p, l); q++) {
                const int n0 = l + 2 * q;
                const float a0 = axial_entry(p, l, k, n0), a1 = axial_entry(p, l, k, n0 + 1);
                t.push_back(make_float4(a0, a0, a1, a1));
            }
        }
    return t;
}

const std::vector<float4> &f32_pair_tables_cached(int p) {
    static std::mutex mu;
    static std::vector<float4> cache[FMM_MAX_P + 1];
    static bool ready[FMM_MAX_P + 1] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (!ready[p]) {
        cache[p] = f32_pair_tables(p);
        ready[p] = true;
    }
    return cache[p];
}

template <int P>
cudaError_t attr_f32() {
    cudaError_t e = allow_max_smem((const void *)k_m2l_rot_f32<P>, VSplit<P>::SMEM);
    return e == cudaSuccess ? allow_max_smem((const void *)k_b_m2l_rot_f32<P>, VSplit<P>::SMEM) : e;
}

template <int P>
void launch_b_f32(const BatchSys *S, const int32_t *off, int nsys, int64_t nchunks, const void *tab,
                  cudaStream_t st) {
    FMM_LAUNCH(k_b_m2l_rot_f32<P>, (unsigned)std::max<int64_t>(1, std::min<int64_t>(nchunks, (int64_t)sm_count() * 3)),
               kF32Threads, VSplit<P>::SMEM, st, S, off, nsys, (const float4 *)tab);
}

template <int P>
cudaError_t launch_f32(Plan &Pl, int64_t tot) {
    const int64_t chunks = (tot + kF32Threads - 1) / kF32Threads;
    FMM_LAUNCH(k_m2l_rot_f32<P>, (unsigned)std::min<int64_t>(chunks, (int64_t)sm_count() * 3), kF32Threads, VSplit<P>::SMEM, Pl.stream, pair_table(Pl), Pl.box_cf, Pl.Mf, Pl.Lh,
               (const float4 *)Pl.f32_tab);
    return cudaGetLastError();
}

}  // namespace

bool m2l_f32_supported(int p) {
    return p == 4 || p == 6 || p == 8 || p == 10 || p == 12 || p == 14 || p == 16;
}

// plan-time setup, so that evaluations are safe to capture into a graph
cudaError_t m2l_f32_setup(Plan &P) {
    // the SIMT float kernel by default; the tensor-core kernel on request, and
    // for orders without a SIMT instance
    const bool tc = m2l_tc_supported(P.p) && (P.tc_m2l_opt || !m2l_f32_supported(P.p));
    if (!tc && !m2l_f32_supported(P.p)) return cudaSuccess;  // FP64 M2L
    P.Mf = (float2 *)palloc(P, (size_t)P.nbox * mf_stride(P.p) * sizeof(float2));
    P.Lh = (double2 *)palloc(P, (size_t)P.nbox * P.nc * sizeof(double2));
    if (!P.Mf || !P.Lh || !P.box_cf) return cudaErrorMemoryAllocation;
    if (tc) {
        P.m2l_tc = true;
        return m2l_tc_setup(P);
    }
    const std::vector<float4> &pt = f32_pair_tables_cached(P.p);
    P.f32_tab = palloc(P, pt.size() * sizeof(float4));
    if (!P.f32_tab) return cudaErrorMemoryAllocation;
    // stream-ordered copy from pageable memory completes before return
    cudaError_t e = cudaMemcpyAsync(P.f32_tab, pt.data(), pt.size() * sizeof(float4), cudaMemcpyHostToDevice, P.stream);
    if (e != cudaSuccess) return e;
    switch (P.p) {
        case 4: return attr_f32<4>();
        case 6: return attr_f32<6>();
        case 8: return attr_f32<8>();
        case 10: return attr_f32<10>();
        case 12: return attr_f32<12>();
        case 14: return attr_f32<14>();
        case 16: return attr_f32<16>();
        default: return cudaSuccess;
    }
}

// single-precision M2L over all levels; leaves the unscaled result in L
cudaError_t m2l_f32_all(Plan &P) {
    const int64_t total = P.nbox * P.nc;
    const unsigned grid = (unsigned)std::min<int64_t>((P.nbox + 7) / 8, (int64_t)sm_count() * 16);  // 8 boxes (warps) per block
    FMM_LAUNCH(k_scale_multipoles, grid, 256, 0, P.stream, P.nbox, P.p, P.radius, P.M, P.Mf);
    cudaMemsetAsync(P.Lh, 0, (size_t)total * sizeof(double2), P.stream);
    const int64_t tot = total_weak(P);
    cudaError_t e = cudaSuccess;
    if (tot > 0 && P.m2l_tc) {
        e = m2l_tc_launch(P);
    } else if (tot > 0) {
        switch (P.p) {
            case 4: e = launch_f32<4>(P, tot); break;
            case 6: e = launch_f32<6>(P, tot); break;
            case 8: e = launch_f32<8>(P, tot); break;
            case 10: e = launch_f32<10>(P, tot); break;
            case 12: e = launch_f32<12>(P, tot); break;
            case 14: e = launch_f32<14>(P, tot); break;
            case 16: e = launch_f32<16>(P, tot); break;
            default: return cudaErrorInvalidValue;
        }
    }
    if (e != cudaSuccess) return e;
    FMM_LAUNCH(k_unscale_locals, grid, 256, 0, P.stream, P.nbox, P.p, P.radius, P.Lh, P.L);
    return cudaGetLastError();
}

// ---- batched stages (every system of a batch in one launch per stage)
cudaError_t batch_m2m_up(const BatchSys *S, const int32_t *off, int nsys, int64_t blocks, int p,
                         const float2 *tab, cudaStream_t st) {
    if (blocks == 0) return cudaGetLastError();
    FMM_LAUNCH(k_b_m2m_up, (unsigned)blocks, 32 * kWarpChildMax, warp_child_smem(p, kWarpChildMax), st, S, off, nsys,
               p, tab);
    return cudaGetLastError();
}

cudaError_t batch_m2l(const BatchSys *S, const int32_t *off, int nsys, int64_t nchunks, int p, const void *tab,
                      cudaStream_t st) {
    if (nchunks == 0) return cudaGetLastError();
    switch (p) {
        case 4: launch_b_f32<4>(S, off, nsys, nchunks, tab, st); break;
        case 6: launch_b_f32<6>(S, off, nsys, nchunks, tab, st); break;
        case 8: launch_b_f32<8>(S, off, nsys, nchunks, tab, st); break;
        case 10: launch_b_f32<10>(S, off, nsys, nchunks, tab, st); break;
        case 12: launch_b_f32<12>(S, off, nsys, nchunks, tab, st); break;
        case 14: launch_b_f32<14>(S, off, nsys, nchunks, tab, st); break;
        case 16: launch_b_f32<16>(S, off, nsys, nchunks, tab, st); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t batch_l2l_down(const BatchSys *S, const int32_t *off, int nsys, int64_t nchunks, int p,
                           const double *tab, const float2 *tab_df, unsigned long long *next, cudaStream_t st) {
    if (nchunks == 0) return cudaGetLastError();
    const unsigned grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((nchunks + kWarpChildMax - 1) / kWarpChildMax, (int64_t)sm_count() * 8));
    FMM_LAUNCH(k_b_l2l_down, grid, 32 * kWarpChildMax, warp_child_smem(p, kWarpChildMax), st, S, off, nsys, p, tab,
               tab_df, next, g_wait_limit.load(), g_withhold.load());
    return cudaGetLastError();
}

cudaError_t batch_smem_limits(int p) {
    const size_t need = warp_child_smem(p, kWarpChildMax);
    cudaError_t e = allow_max_smem((const void *)k_b_m2m_up, need);
    return e == cudaSuccess ? allow_max_smem((const void *)k_b_l2l_down, need) : e;
}

}  // namespace fmm

extern "C" int64_t fmm_set_wait_limit(int64_t sleeps, int64_t withhold) {
    const long long prev = fmm::g_wait_limit.load();
    fmm::g_wait_limit.store(sleeps > 0 ? sleeps : (1LL << 24));
    fmm::g_withhold.store(withhold > 0 ? withhold : -1);
    return (int64_t)prev;
}
