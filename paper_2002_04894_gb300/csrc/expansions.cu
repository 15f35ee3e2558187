// Expansion stages of Algorithm 1 in double precision: P2M at the leaves,
// M2M upward (Algorithm 1), M2L at every level with weak pairs and L2L
// downward (Algorithm 3), and L2P at the leaves (Algorithm 4).
//
// Expansions are spherical-harmonic multipole and local series of order p
// about the cell centres (Sec. 2.1). With Y_n^m = (-1)^m R_n^m (m >= 0),
// Y_n^{-m} = conj(R_n^m), R_n^m = r^n P_n^m e^{im phi}/(n+m)! and the matching
// irregular Th_n^m built from I_n^m = (n-m)! P_n^m e^{im phi}/r^{n+1}:
//   M_n^m  = sum_j q_j conj(Y_n^m(x_j - c))                         (P2M)
//   M'_n^m = sum_{k,l} conj(Y_k^l(c - c')) M_{n-k}^{m-l}             (M2M)
//   L_k^l  = (-1)^k sum_{n,m} M_n^m Th_{n+k}^{m+l}(c_t - c_s)        (M2L)
//   L'_j^i = sum_{k>=j,l} L_k^l conj(Y_{k-j}^{l-i}(c' - c))          (L2L)
//   phi(c + s) = sum_{k,l} L_k^l conj(Y_k^l(s)), E = -grad phi        (L2P)
// Only m >= 0 is stored: real charges give C_n^{-m} = (-1)^m conj(C_n^m).
//
// GPU mapping: P2M is one CTA per leaf with one point per lane, streaming the
// harmonics through the Legendre recurrences and reducing each coefficient
// over the warp; M2M, L2L and M2L (in m2l.cu) use the rotational form, one
// translation per thread; L2P is one thread per point with O(1) registers
// (the series and its gradient accumulate as the recurrence runs).

#include <algorithm>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int kExpThreads = 128;

template <typename T>
__global__ void k_gather_q(const T *__restrict__ qin, const int32_t *__restrict__ perm,
                           double *__restrict__ q, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        q[i] = (double)qin[perm[i]];
}

__global__ void __launch_bounds__(kExpThreads)
k_p2m(int B, int p, const double *__restrict__ x, const double *__restrict__ y,
      const double *__restrict__ z, const double *__restrict__ q, const int32_t *__restrict__ begin,
      const int32_t *__restrict__ count, const double *__restrict__ centre, double2 *__restrict__ M) {
    extern __shared__ double2 acc[];  // [warps][nc]
    const int nc = ncoef(p);
    const int64_t g = ((int64_t)1 << B) - 1 + blockIdx.x;
    const int b = begin[g], n = count[g];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const double cx = centre[3 * g], cy = centre[3 * g + 1], cz = centre[3 * g + 2];
    for (int c = threadIdx.x; c < nc * (kExpThreads / 32); c += kExpThreads)
        acc[c] = make_double2(0.0, 0.0);
    __syncthreads();
    double2 *mine = acc + w * nc;
    for (int base = w * 32; base < n; base += kExpThreads) {
        const int i = base + lane;
        const bool valid = i < n;
        const double dx = valid ? x[b + i] - cx : 0.0;
        const double dy = valid ? y[b + i] - cy : 0.0;
        const double dz = valid ? z[b + i] - cz : 0.0;
        const double qi = valid ? q[b + i] : 0.0;
        const double r2 = dx * dx + dy * dy + dz * dz;
        double2 mm = make_double2(1.0, 0.0);  // R_m^m
        for (int m = 0; m <= p; m++) {
            if (m > 0) mm = cscale(cmul(mm, make_double2(dx, dy)), 0.5 / m);
            double2 cur = mm, prev = make_double2(0.0, 0.0);
            const double sg = (m & 1) ? -qi : qi;
            for (int nn = m; nn <= p; nn++) {
                if (nn > m) {
                    double2 nxt;
                    if (nn == m + 1) {
                        nxt = cscale(cur, dz);
                    } else {
                        const double s = 1.0 / ((double)(nn - m) * (double)(nn + m));
                        nxt = make_double2(((2 * nn - 1) * dz * cur.x - r2 * prev.x) * s,
                                           ((2 * nn - 1) * dz * cur.y - r2 * prev.y) * s);
                    }
                    prev = cur;
                    cur = nxt;
                }
                // q conj(Y_n^m) = q (-1)^m conj(R_n^m)
                double vr = sg * cur.x, vi = -sg * cur.y;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    vr += __shfl_xor_sync(0xffffffffu, vr, o);
                    vi += __shfl_xor_sync(0xffffffffu, vi, o);
                }
                if (lane == 0) {
                    double2 a = mine[tri(nn, m)];
                    mine[tri(nn, m)] = make_double2(a.x + vr, a.y + vi);
                }
            }
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nc; c += kExpThreads) {
        double2 s = make_double2(0.0, 0.0);
        for (int j = 0; j < kExpThreads / 32; j++) s = cadd(s, acc[j * nc + c]);
        M[g * nc + c] = s;
    }
}

// L2P: far-field potential and field at every leaf point (leaf order)
__global__ void __launch_bounds__(kExpThreads)
k_l2p(int B, int p, int64_t npts, const double *__restrict__ x, const double *__restrict__ y,
      const double *__restrict__ z, const int32_t *__restrict__ begin,
      const int32_t *__restrict__ count, const double *__restrict__ centre,
      const double2 *__restrict__ L, double *__restrict__ far_phi, double *__restrict__ far_E) {
    extern __shared__ double2 Ls[];
    const int nc = ncoef(p);
    const int64_t g = ((int64_t)1 << B) - 1 + blockIdx.x;
    const int b = begin[g], n = count[g];
    for (int c = threadIdx.x; c < nc; c += kExpThreads) Ls[c] = L[g * nc + c];
    __syncthreads();
    const double cx = centre[3 * g], cy = centre[3 * g + 1], cz = centre[3 * g + 2];
    for (int i = threadIdx.x; i < n; i += kExpThreads) {
        const double dx = x[b + i] - cx, dy = y[b + i] - cy, dz = z[b + i] - cz;
        const double r2 = dx * dx + dy * dy + dz * dz;
        double phi = 0.0, g0 = 0.0;          // phi and the degree-1, order-0 shifted coefficient
        double2 g1 = make_double2(0.0, 0.0); // degree-1, order-1 shifted coefficient
        double2 mm = make_double2(1.0, 0.0);
        for (int m = 0; m <= p; m++) {
            if (m > 0) mm = cscale(cmul(mm, make_double2(dx, dy)), 0.5 / m);
            double2 cur = mm, prev = make_double2(0.0, 0.0);
            const double w = m == 0 ? 1.0 : 2.0;
            for (int nn = m; nn <= p; nn++) {
                if (nn > m) {
                    double2 nxt;
                    if (nn == m + 1) {
                        nxt = cscale(cur, dz);
                    } else {
                        const double s = 1.0 / ((double)(nn - m) * (double)(nn + m));
                        nxt = make_double2(((2 * nn - 1) * dz * cur.x - r2 * prev.x) * s,
                                           ((2 * nn - 1) * dz * cur.y - r2 * prev.y) * s);
                    }
                    prev = cur;
                    cur = nxt;
                }
                // Y = (-1)^m R; Yc = conj(Y)
                const double2 Y = (m & 1) ? make_double2(-cur.x, -cur.y) : cur;
                const double2 Yc = cconj(Y);
                phi += w * cmul(Ls[tri(nn, m)], Yc).x;
                if (nn < p) {
                    g0 += w * cmul(Ls[tri(nn + 1, m)], Yc).x;
                    g1 = cadd(g1, cmul(Ls[tri(nn + 1, m + 1)], Yc));
                    if (m >= 1) {
                        const double2 t = cmul(cconj(Ls[tri(nn + 1, m - 1)]), Y);
                        g1 = make_double2(g1.x - t.x, g1.y - t.y);
                    }
                }
            }
        }
        far_phi[b + i] = phi;
        far_E[b + i] = g1.x;
        far_E[npts + b + i] = g1.y;
        far_E[2 * npts + b + i] = -g0;
    }
}

}  // namespace

// the first level with weak pairs: multipoles above it are never read (no
// M2L there, and M2M into them would only feed unused levels), so they are
// left zero unless the plan forms every level (a rank of a split system
// sends its root's multipole); local expansions above it are exactly zero
int first_weak_level_of(const Plan &P) {
    int lw = P.B + 1;
    for (int l = P.B; l >= 1; l--)
        if (P.nweak[l] > 0) lw = l;
    return lw;
}

static int first_weak_level(const Plan &P) {
    int lw = P.B + 1;
    for (int l = P.B; l >= 1; l--)
        if (P.nweak[l] > 0) lw = l;
    return P.full_upward ? 0 : lw;
}

// Binary trees of up to kOneLaunchMaxLevels levels run the upward and
// downward passes as one launch each (a warp walking up from each leaf; a
// queue of boxes with bounded waits on the parent); deeper trees run one
// launch per level, which keeps the FP64 pipe busier on the large levels
// (measured on 8M points at 17 levels: M2M 7.4 ms per level against 9.6 ms
// in one launch, L2L 6.9 against 8.2 ms) while the launches of the small
// levels no longer matter.
constexpr int kOneLaunchMaxLevels = 13;
static bool one_launch_passes(const Plan &P) { return P.step == 1 && P.B <= kOneLaunchMaxLevels; }

// P2M and M2M (Algorithm 1)
cudaError_t eval_upward(Plan &P, const void *charges, int dtype) {
    cudaStream_t st = P.stream;
    const int64_t n = P.n;
    const int nc = P.nc;
    const bool mixed = P.prec == FMM_PREC_MIXED;
    const int gq = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
    stage_mark(P, FMM_STAGE_P2M, 0);
    if (mixed) {
        cudaError_t e = mixed_p2m(P, charges, dtype);
        if (e != cudaSuccess) return e;
    } else {
        if (dtype == FMM_F64)
            FMM_LAUNCH(k_gather_q<double>, gq, 256, 0, st, (const double *)charges, P.perm, P.q, n);
        else
            FMM_LAUNCH(k_gather_q<float>, gq, 256, 0, st, (const float *)charges, P.perm, P.q, n);
        FMM_LAUNCH(k_p2m, (unsigned)P.nleaf, kExpThreads, sizeof(double2) * nc * (kExpThreads / 32),
                   st, P.B, P.p, P.x, P.y, P.z, P.q, P.begin, P.count, P.centre, P.M);
    }
    stage_mark(P, FMM_STAGE_P2M, 1);
    const int lw = first_weak_level(P);
    // with 2^step children per box only every step-th bisection level holds
    // expansions; the levels in between stay zero
    const int sp = P.step;
    stage_mark(P, FMM_STAGE_M2M, 0);
    if (one_launch_passes(P)) {
        m2m_up(P, std::min(lw, P.B));
    } else {
        for (int pl = P.B - 1; pl >= 0; pl--) {
            if (pl % sp == 0 && pl >= lw)
                m2m_level(P, pl + sp);
            else
                cudaMemsetAsync(P.M + (((int64_t)1 << pl) - 1) * nc, 0,
                                (size_t)((int64_t)1 << pl) * nc * sizeof(double2), st);
        }
    }
    stage_mark(P, FMM_STAGE_M2M, 1);
    return cudaGetLastError();
}

// M2L at every level, then L2L downward (Algorithm 3), then L2P (Algorithm 4).
// Local expansions and near-field terms from outside the plan (a split
// system's other ranks) are added between M2L and L2L and after L2P.
cudaError_t eval_downward(Plan &P) {
    cudaStream_t st = P.stream;
    const int64_t n = P.n;
    const bool mixed = P.prec == FMM_PREC_MIXED;
    const int lw = first_weak_level(P);
    const int sp = P.step;
    stage_mark(P, FMM_STAGE_M2L, 0);
    {
        // all levels in one launch; every L is (re)written, the root's stays zero
        cudaError_t e = (mixed && P.Mf) ? m2l_f32_all(P) : m2l_all(P);
        if (e != cudaSuccess) return e;
        if (P.ext_active) {
            e = add_external_locals(P);
            if (e != cudaSuccess) return e;
        }
    }
    stage_mark(P, FMM_STAGE_M2L, 1);
    stage_mark(P, FMM_STAGE_L2L, 0);
    // L2L into a level whose parents hold nothing would only add zeros
    if (one_launch_passes(P)) {
        l2l_down(P, lw);
    } else {
        for (int l = sp; l <= P.B; l += sp)
            if (l - sp >= lw || P.ext_active) l2l_level(P, l);
    }
    stage_mark(P, FMM_STAGE_L2L, 1);
    stage_mark(P, FMM_STAGE_L2P, 0);
    if (mixed) {
        cudaError_t e = mixed_l2p(P);
        if (e != cudaSuccess) return e;
    } else {
        FMM_LAUNCH(k_l2p, (unsigned)P.nleaf, kExpThreads, sizeof(double2) * P.nc, st, P.B, P.p, n, P.x,
                   P.y, P.z, P.begin, P.count, P.centre, P.L, P.far_phi, P.far_E);
        if (P.ext_active) {
            cudaError_t e = add_external_near(P);
            if (e != cudaSuccess) return e;
        }
    }
    stage_mark(P, FMM_STAGE_L2P, 1);
    return cudaGetLastError();
}

cudaError_t eval_expansions(Plan &P, const void *charges, int dtype) {
    cudaError_t e = eval_upward(P, charges, dtype);
    return e == cudaSuccess ? eval_downward(P) : e;
}

}  // namespace fmm
