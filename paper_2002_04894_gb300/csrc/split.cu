// One rank's part of a system split over several devices (Sec. 2.2 and
// Algorithms 2-4): the plan of the rank's subtree runs its upward pass, hands
// out multipoles and leaf points for the other ranks, takes in theirs (M2L
// from received multipoles, the near field of received points) and finishes
// the downward pass. The bookkeeping (which boxes, which ranks) is the
// caller's; every arithmetic step runs here, in double precision (the plain
// form).

#include <algorithm>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

__global__ void k_gather_boxes(int level, int64_t n, const int32_t *__restrict__ idx, int nc,
                               const double2 *__restrict__ M, double2 *__restrict__ out) {
    const int64_t off = ((int64_t)1 << level) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * nc;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / nc, c = i - b * nc;
        out[i] = M[(off + idx[b]) * nc + c];
    }
}

__global__ void k_add_boxes(int level, int64_t n, const int32_t *__restrict__ idx, int nc,
                            const double2 *__restrict__ in, double2 *Lx) {
    const int64_t off = ((int64_t)1 << level) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * nc;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / nc, c = i - b * nc;
        atomicAdd(&Lx[(off + idx[b]) * nc + c].x, in[i].x);
        atomicAdd(&Lx[(off + idx[b]) * nc + c].y, in[i].y);
    }
}

__global__ void k_add_all(int64_t n, const double *__restrict__ a, double *__restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] += a[i];
}

// points (x, y, z, q) of the given leaves, leaf after leaf, at off[i]
__global__ void k_leaf_points(int B, int64_t n, const int32_t *__restrict__ leaf, const int64_t *__restrict__ off,
                              const int32_t *__restrict__ begin, const int32_t *__restrict__ count,
                              const double *__restrict__ x, const double *__restrict__ y,
                              const double *__restrict__ z, const double *__restrict__ q,
                              double4 *__restrict__ out) {
    const int64_t base = ((int64_t)1 << B) - 1;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const int64_t g = base + leaf[i];
        const int b = begin[g], c = count[g];
        for (int k = threadIdx.x; k < c; k += blockDim.x)
            out[off[i] + k] = make_double4(x[b + k], y[b + k], z[b + k], q[b + k]);
    }
}

// near field of received points at the points of a leaf: pair i is (target
// leaf tgt[i], sources src[off[i] .. off[i + 1])); one block per pair, one
// target per thread; phi, Ex, Ey, Ez (leaf order, SoA) accumulated
__global__ void __launch_bounds__(128)
k_p2p_external(int B, int64_t npts, int64_t n, const int32_t *__restrict__ tgt, const int64_t *__restrict__ off,
               const double4 *__restrict__ src, const int32_t *__restrict__ begin,
               const int32_t *__restrict__ count, const double *__restrict__ x, const double *__restrict__ y,
               const double *__restrict__ z, double *near) {
    __shared__ double4 tile[128];
    const int64_t base = ((int64_t)1 << B) - 1;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const int64_t g = base + tgt[i];
        const int b = begin[g], c = count[g];
        const int64_t s0 = off[i], s1 = off[i + 1];
        for (int t0 = 0; t0 < c; t0 += blockDim.x) {
            const int t = t0 + threadIdx.x;
            const bool active = t < c;
            const double xi = active ? x[b + t] : 0.0, yi = active ? y[b + t] : 0.0, zi = active ? z[b + t] : 0.0;
            double phi = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
            for (int64_t sb = s0; sb < s1; sb += blockDim.x) {
                __syncthreads();
                if (sb + threadIdx.x < s1) tile[threadIdx.x] = src[sb + threadIdx.x];
                __syncthreads();
                const int m = (int)std::min<int64_t>(blockDim.x, s1 - sb);
                for (int j = 0; j < m; j++) {
                    const double4 s = tile[j];
                    const double dx = xi - s.x, dy = yi - s.y, dz = zi - s.z;
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    const double rinv = r2 > 0.0 ? rsqrt(r2) : 0.0;
                    const double qr = s.w * rinv, qr3 = qr * rinv * rinv;
                    phi += qr;
                    ex += qr3 * dx;
                    ey += qr3 * dy;
                    ez += qr3 * dz;
                }
            }
            if (active) {
                atomicAdd(&near[b + t], phi);
                atomicAdd(&near[npts + b + t], ex);
                atomicAdd(&near[2 * npts + b + t], ey);
                atomicAdd(&near[3 * npts + b + t], ez);
            }
        }
    }
}

// ---- explicit translations between boxes outside any plan (the top levels
// of a split tree: a handful of boxes), direct O(p^4) sums, one per thread.
// R_n^m(x) = r^n P_n^m(cos t) e^{im phi} / (n+m)!, I_n^m(x) = (n-m)! P_n^m(cos t)
// e^{im phi} / r^{n+1} (m >= 0, no Condon-Shortley phase) from the Legendre
// recurrences; signed views Y_n^m = (-1)^m R_n^m, Y_n^{-m} = conj(R_n^m), and
// likewise Th from I; real-source coefficients C_n^{-m} = (-1)^m conj(C_n^m).
constexpr int kTrMax = 2 * FMM_MAX_P;

__device__ void solid_regular(double x, double y, double z, int p, double2 *R) {
    const double r2 = x * x + y * y + z * z;
    R[0] = make_double2(1.0, 0.0);
    for (int m = 0; m <= p; m++) {
        if (m > 0) R[tri(m, m)] = cscale(cmul(make_double2(x, y), R[tri(m - 1, m - 1)]), 0.5 / m);
        if (m + 1 <= p) R[tri(m + 1, m)] = cscale(R[tri(m, m)], z);
        for (int n = m + 2; n <= p; n++) {
            const double2 a = R[tri(n - 1, m)], b = R[tri(n - 2, m)];
            const double s = 1.0 / ((double)(n - m) * (double)(n + m));
            R[tri(n, m)] = make_double2(((2 * n - 1) * z * a.x - r2 * b.x) * s, ((2 * n - 1) * z * a.y - r2 * b.y) * s);
        }
    }
}

__device__ void solid_irregular(double x, double y, double z, int p, double2 *Ir) {
    const double r2 = x * x + y * y + z * z, ir2 = 1.0 / r2;
    Ir[0] = make_double2(sqrt(ir2), 0.0);
    for (int m = 0; m <= p; m++) {
        if (m > 0) Ir[tri(m, m)] = cscale(cmul(make_double2(x, y), Ir[tri(m - 1, m - 1)]), (2.0 * m - 1.0) * ir2);
        if (m + 1 <= p) Ir[tri(m + 1, m)] = cscale(Ir[tri(m, m)], (2.0 * m + 1.0) * z * ir2);
        for (int n = m + 2; n <= p; n++) {
            const double2 a = Ir[tri(n - 1, m)], b = Ir[tri(n - 2, m)];
            const double c = (double)(n - 1 + m) * (double)(n - 1 - m);
            Ir[tri(n, m)] = make_double2(((2 * n - 1) * z * a.x - c * b.x) * ir2, ((2 * n - 1) * z * a.y - c * b.y) * ir2);
        }
    }
}

__device__ __forceinline__ double2 signed_harm(const double2 *H, int n, int m) {
    if (n < 0 || m > n || -m > n) return make_double2(0.0, 0.0);
    if (m >= 0) return (m & 1) ? make_double2(-H[tri(n, m)].x, -H[tri(n, m)].y) : H[tri(n, m)];
    return cconj(H[tri(n, -m)]);
}

// kind 0 M2M (src multipole about cs -> multipole about cd), 1 M2L (multipole
// about cs -> local about cd), 2 L2L (local about cs -> local about cd); the
// result is added to dst
__global__ void k_translate(int kind, int p, int64_t n, const double2 *__restrict__ src,
                            const double *__restrict__ cs, const double *__restrict__ cd, double2 *dst) {
    double2 H[(kTrMax + 1) * (kTrMax + 2) / 2];
    const int nc = ncoef(p);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 *C = src + i * nc;
        double2 *D = dst + i * nc;
        const double dx = cd[3 * i] - cs[3 * i], dy = cd[3 * i + 1] - cs[3 * i + 1], dz = cd[3 * i + 2] - cs[3 * i + 2];
        if (kind == 1) {
            solid_irregular(dx, dy, dz, 2 * p, H);
            for (int k = 0; k <= p; k++)
                for (int l = 0; l <= k; l++) {
                    double2 s = make_double2(0.0, 0.0);
                    for (int nn = 0; nn <= p; nn++)
                        for (int m = -nn; m <= nn; m++) s = cadd(s, cmul(coef_at(C, nn, m), signed_harm(H, nn + k, m + l)));
                    if (k & 1) s = make_double2(-s.x, -s.y);
                    D[tri(k, l)] = cadd(D[tri(k, l)], s);
                }
        } else {
            // M2M: offset child - parent = cs - cd; L2L: offset child - parent = cd - cs
            if (kind == 0)
                solid_regular(-dx, -dy, -dz, p, H);
            else
                solid_regular(dx, dy, dz, p, H);
            for (int j = 0; j <= p; j++)
                for (int a = 0; a <= j; a++) {
                    double2 s = make_double2(0.0, 0.0);
                    if (kind == 0) {
                        for (int k = 0; k <= j; k++)
                            for (int l = -k; l <= k; l++)
                                s = cadd(s, cmul(cconj(signed_harm(H, k, l)), coef_at(C, j - k, a - l)));
                    } else {
                        for (int k = j; k <= p; k++)
                            for (int l = -k; l <= k; l++)
                                s = cadd(s, cmul(coef_at(C, k, l), cconj(signed_harm(H, k - j, l - a))));
                    }
                    D[tri(j, a)] = cadd(D[tri(j, a)], s);
                }
        }
    }
}

unsigned grid_for(int64_t work) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)sm_count() * 8)); }

}  // namespace

cudaError_t add_external_locals(Plan &P) {
    const int64_t n = P.nbox * P.nc * 2;
    FMM_LAUNCH(k_add_all, grid_for(n), 256, 0, P.stream, n, (const double *)P.L_ext, (double *)P.L);
    return cudaGetLastError();
}

cudaError_t add_external_near(Plan &P) {
    // far_phi and far_E are consecutive in the plan's layout only by chance;
    // add them separately
    FMM_LAUNCH(k_add_all, grid_for(P.n), 256, 0, P.stream, P.n, P.near_ext, P.far_phi);
    FMM_LAUNCH(k_add_all, grid_for(3 * P.n), 256, 0, P.stream, 3 * P.n, P.near_ext + P.n, P.far_E);
    return cudaGetLastError();
}

}  // namespace fmm

using fmm::Plan;
using fmm::cuda_status;

namespace {
bool dev(const void *p) { return fmm::ptr_kind(p) == 1; }
bool split_plan(fmm_plan_t plan) { return plan && plan->P.prec == FMM_PREC_FP64; }
}  // namespace

extern "C" {

int fmm_theta_test(double theta, int64_t n, const double *ca, const double *ra, const double *cb,
                   const double *rb, uint8_t *weak, void *stream) {
    if (n < 0 || !(theta >= 0.0 && theta < 1.0)) return FMM_EINVAL;
    if (n == 0) return FMM_OK;
    if (!dev(ca) || !dev(ra) || !dev(cb) || !dev(rb) || !dev(weak)) return FMM_EINVAL;
    return cuda_status(fmm::theta_pairs(theta, n, ca, ra, cb, rb, weak, (cudaStream_t)stream));
}

int fmm_translate(int kind, int p, int64_t n, const double *src, const double *csrc, const double *cdst,
                  double *dst, void *stream) {
    if (kind < 0 || kind > 2 || p < 0 || p > FMM_MAX_P || n < 0) return FMM_EINVAL;
    if (n == 0) return FMM_OK;
    if (!dev(src) || !dev(csrc) || !dev(cdst) || !dev(dst)) return FMM_EINVAL;
    FMM_LAUNCH(fmm::k_translate, (unsigned)((n + 31) / 32), 32, 0, (cudaStream_t)stream, kind, p, n,
               (const double2 *)src, csrc, cdst, (double2 *)dst);
    return cuda_status(cudaGetLastError());
}

int fmm_eval_upward(fmm_plan_t plan, const void *charges, void *stream) {
    if (!split_plan(plan) || !dev(charges)) return FMM_EINVAL;
    Plan &P = plan->P;
    P.stream = (cudaStream_t)stream;
    if (!P.L_ext) {
        P.L_ext = (double2 *)fmm::palloc(P, (size_t)P.nbox * P.nc * sizeof(double2));
        P.near_ext = (double *)fmm::palloc(P, (size_t)P.n * 4 * sizeof(double));
        if (!P.L_ext || !P.near_ext) return FMM_ENOMEM;
    }
    P.full_upward = true;
    P.ext_active = true;
    cudaMemsetAsync(P.L_ext, 0, (size_t)P.nbox * P.nc * sizeof(double2), P.stream);
    cudaMemsetAsync(P.near_ext, 0, (size_t)P.n * 4 * sizeof(double), P.stream);
    return cuda_status(fmm::eval_upward(P, charges, P.dtype));
}

int fmm_plan_multipoles(fmm_plan_t plan, int level, int64_t n, const int32_t *idx, double *out, void *stream) {
    if (!split_plan(plan) || level < 0 || level > plan->P.B || n < 0) return FMM_EINVAL;
    if (n == 0) return FMM_OK;
    if (!dev(idx) || !dev(out)) return FMM_EINVAL;
    Plan &P = plan->P;
    FMM_LAUNCH(fmm::k_gather_boxes, fmm::grid_for(n * P.nc), 256, 0, (cudaStream_t)stream, level, n, idx, P.nc,
               P.M, (double2 *)out);
    return cuda_status(cudaGetLastError());
}

int fmm_plan_add_locals(fmm_plan_t plan, int level, int64_t n, const int32_t *idx, const double *L, void *stream) {
    if (!split_plan(plan) || !plan->P.L_ext || level < 0 || level > plan->P.B || n < 0) return FMM_EINVAL;
    if (n == 0) return FMM_OK;
    if (!dev(idx) || !dev(L)) return FMM_EINVAL;
    Plan &P = plan->P;
    FMM_LAUNCH(fmm::k_add_boxes, fmm::grid_for(n * P.nc), 256, 0, (cudaStream_t)stream, level, n, idx, P.nc,
               (const double2 *)L, P.L_ext);
    return cuda_status(cudaGetLastError());
}

int fmm_m2l_external(fmm_plan_t plan, int level, int64_t n, const int32_t *tgt, const double *M,
                     const double *centre, void *stream) {
    if (!split_plan(plan) || !plan->P.L_ext || level < 0 || level > plan->P.B || n < 0) return FMM_EINVAL;
    if (n == 0) return FMM_OK;
    if (!dev(tgt) || !dev(M) || !dev(centre)) return FMM_EINVAL;
    Plan &P = plan->P;
    P.stream = (cudaStream_t)stream;
    return cuda_status(fmm::m2l_external(P, level, n, tgt, (const double2 *)M, centre));
}

int fmm_plan_leaf_points(fmm_plan_t plan, int64_t n, const int32_t *leaf, const int64_t *off, double *out,
                         void *stream) {
    if (!split_plan(plan) || n < 0) return FMM_EINVAL;
    if (n == 0) return FMM_OK;
    if (!dev(leaf) || !dev(off) || !dev(out)) return FMM_EINVAL;
    Plan &P = plan->P;
    FMM_LAUNCH(fmm::k_leaf_points, (unsigned)std::min<int64_t>(n, (int64_t)fmm::sm_count() * 8), 128, 0,
               (cudaStream_t)stream, P.B, n, leaf, off, P.begin, P.count, P.x, P.y, P.z, P.q, (double4 *)out);
    return cuda_status(cudaGetLastError());
}

int fmm_p2p_external(fmm_plan_t plan, int64_t n, const int32_t *tgt, const int64_t *off, const double *src,
                     void *stream) {
    if (!split_plan(plan) || !plan->P.near_ext || n < 0) return FMM_EINVAL;
    if (n == 0) return FMM_OK;
    if (!dev(tgt) || !dev(off) || !dev(src)) return FMM_EINVAL;
    Plan &P = plan->P;
    FMM_LAUNCH(fmm::k_p2p_external, (unsigned)std::min<int64_t>(n, (int64_t)fmm::sm_count() * 8), 128, 0,
               (cudaStream_t)stream, P.B, P.n, n, tgt, off, (const double4 *)src, P.begin, P.count, P.x, P.y, P.z,
               P.near_ext);
    return cuda_status(cudaGetLastError());
}

int fmm_eval_downward(fmm_plan_t plan, void *potentials, void *fields, void *stream) {
    if (!split_plan(plan) || !plan->P.ext_active || !dev(potentials) || (fields && !dev(fields)))
        return FMM_EINVAL;
    Plan &P = plan->P;
    P.stream = (cudaStream_t)stream;
    cudaError_t e = fmm::eval_downward(P);
    if (e == cudaSuccess) e = fmm::eval_p2p(P, potentials, fields, P.dtype);
    P.full_upward = false;
    P.ext_active = false;
    return cuda_status(e);
}

}  // extern "C"
