// Near field (P2P, Algorithm 4) and the exact sum of Eq. 2.1.
//
// P2P: for every target leaf, the direct interaction with the points of all
// strongly connected leaves (itself included), pairs at zero distance
// skipped. One CTA per work unit (a tile of a target leaf's points against a
// segment of its strong list), one target point per thread; source leaves
// are staged through shared memory in tiles of (x, y, z, q). The kernel adds
// the far field left by L2P and writes phi and E straight to the caller's
// arrays in input order (the un-permute step); a leaf whose strong list was
// cut into segments leaves per-segment partial sums instead, which the
// combine pass adds in segment order.
//
// Direct: one CTA per target, threads stride over all sources with
// Neumaier-compensated partial sums, then a block reduction.

#include <algorithm>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int kP2PThreads = 128;

template <typename OutT>
__global__ void __launch_bounds__(kP2PThreads)
k_p2p_f64(int B, int64_t npts, const double *__restrict__ x, const double *__restrict__ y,
          const double *__restrict__ z, const double *__restrict__ q,
          const int32_t *__restrict__ begin, const int32_t *__restrict__ count,
          const int32_t *__restrict__ ssrc, const int4 *__restrict__ units, const int32_t *__restrict__ upart,
          const int32_t *__restrict__ nunits, const int32_t *__restrict__ perm,
          const double *__restrict__ far_phi, const double *__restrict__ far_E, double4 *__restrict__ partial,
          OutT *__restrict__ pot, OutT *__restrict__ field) {
    struct alignas(16) Src {
        double x, y, z, q;
    };
    __shared__ Src tile[kP2PThreads];
    const int64_t off = ((int64_t)1 << B) - 1;
    static_assert(kP2PThreads == kP2PTile, "one target per thread");
    if ((int)blockIdx.x >= *nunits) return;  // launched for an upper bound on the units
    const int4 unit = units[blockIdx.x];
    const int part = upart[blockIdx.x];
    const int t = unit.x;
    const int bt = begin[off + t], nt = count[off + t];
    const int e0 = unit.z, e1 = unit.w;  // this unit's segment of the strong list
    {
        const int tb = unit.y;
        const int i = tb + threadIdx.x;
        const bool active = i < nt;
        // a warp with no target of the unit stages sources and keeps the
        // barriers, but skips the products (small leaves: the warps past the
        // leaf's last target cost no arithmetic)
        const bool busy = __any_sync(0xffffffffu, active);  // warp-uniform
        const double xi = active ? x[bt + i] : 0.0;
        const double yi = active ? y[bt + i] : 0.0;
        const double zi = active ? z[bt + i] : 0.0;
        double phi = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
        for (int e = e0; e < e1; e++) {
            const int64_t gs = off + ssrc[e];
            const int bs = begin[gs], ns = count[gs];
            for (int sb = 0; sb < ns; sb += kP2PThreads) {
                const int j = sb + threadIdx.x;
                tile[threadIdx.x] = j < ns ? Src{x[bs + j], y[bs + j], z[bs + j], q[bs + j]} : Src{0.0, 0.0, 0.0, 0.0};
                __syncthreads();
                const int mcount = min(kP2PThreads, ns - sb);
                for (int jj = 0; jj < (busy ? mcount : 0); jj++) {
                    const Src s = tile[jj];
                    const double dx = xi - s.x, dy = yi - s.y, dz = zi - s.z;
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    const double rinv = r2 > 0.0 ? rsqrt(r2) : 0.0;
                    const double qr = s.q * rinv;
                    const double qr3 = qr * rinv * rinv;
                    phi += qr;
                    ex += qr3 * dx;
                    ey += qr3 * dy;
                    ez += qr3 * dz;
                }
                __syncthreads();
            }
        }
        if (active && part >= 0) {  // one segment of a split leaf: its partial sums
            partial[part + i] = make_double4(phi, ex, ey, ez);
        } else if (active) {
            const int64_t a = bt + i;
            const int64_t o = perm[a];
            pot[o] = (OutT)(far_phi[a] + phi);
            if (field) {
                field[3 * o] = (OutT)(far_E[a] + ex);
                field[3 * o + 1] = (OutT)(far_E[npts + a] + ey);
                field[3 * o + 2] = (OutT)(far_E[2 * npts + a] + ez);
            }
        }
    }
}

__device__ __forceinline__ void neumaier(double &s, double &c, double v) {
    const double t = s + v;
    if (fabs(s) >= fabs(v))
        c += (s - t) + v;
    else
        c += (v - t) + s;
    s = t;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_direct(const T *__restrict__ pts, const T *__restrict__ q, int64_t n,
         const int64_t *__restrict__ targets, T *__restrict__ pot, T *__restrict__ field) {
    __shared__ double red[4][256];
    const int64_t i = targets[blockIdx.x];
    if (i < 0 || i >= n) {  // out-of-range index: NaN outputs, no access
        if (threadIdx.x < 4) {
            const T nan = (T)__longlong_as_double(0x7ff8000000000000ll);
            if (threadIdx.x == 0)
                pot[blockIdx.x] = nan;
            else if (field)
                field[3 * blockIdx.x + threadIdx.x - 1] = nan;
        }
        return;
    }
    const double xi = (double)pts[3 * i], yi = (double)pts[3 * i + 1], zi = (double)pts[3 * i + 2];
    double s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
    for (int64_t j = threadIdx.x; j < n; j += 256) {
        const double dx = xi - (double)pts[3 * j], dy = yi - (double)pts[3 * j + 1],
                     dz = zi - (double)pts[3 * j + 2];
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 == 0.0) continue;
        const double r = sqrt(r2);
        const double qj = (double)q[j];
        const double qr3 = qj / (r2 * r);
        neumaier(s[0], c[0], qj / r);
        neumaier(s[1], c[1], qr3 * dx);
        neumaier(s[2], c[2], qr3 * dy);
        neumaier(s[3], c[3], qr3 * dz);
    }
    for (int a = 0; a < 4; a++) red[a][threadIdx.x] = s[a] + c[a];
    __syncthreads();
    if (threadIdx.x < 4) {
        double ss = 0.0, cc = 0.0;
        for (int j = 0; j < 256; j++) neumaier(ss, cc, red[threadIdx.x][j]);
        const double v = ss + cc;
        if (threadIdx.x == 0)
            pot[blockIdx.x] = (T)v;
        else if (field)
            field[3 * blockIdx.x + threadIdx.x - 1] = (T)v;
    }
}

// Finishes the leaves whose strong list was cut into segments: per target,
// the segments' partial sums added in segment order, then the far field;
// outputs in input order. Leaves without partial slots are skipped.
template <typename OutT, typename FarT>
__global__ void __launch_bounds__(128)
k_p2p_combine(int B, int64_t npts, const int32_t *__restrict__ begin, const int32_t *__restrict__ count,
              const int32_t *__restrict__ poff, const double4 *__restrict__ partial,
              const int32_t *__restrict__ perm, const FarT *__restrict__ far_phi, const FarT *__restrict__ far_E,
              OutT *__restrict__ pot, OutT *__restrict__ field) {
    const int64_t nl = (int64_t)1 << B;
    for (int64_t t = blockIdx.x; t < nl; t += gridDim.x) {
        const int p0 = poff[t], np = poff[t + 1] - p0;
        if (np == 0) continue;
        const int nt = count[nl - 1 + t], bt = begin[nl - 1 + t];
        const int k = np / nt;
        for (int i = threadIdx.x; i < nt; i += blockDim.x) {
            double4 s = partial[p0 + i];
            for (int j = 1; j < k; j++) {
                const double4 v = partial[p0 + j * nt + i];
                s.x += v.x;
                s.y += v.y;
                s.z += v.z;
                s.w += v.w;
            }
            const int64_t a = bt + i;
            const int64_t o = perm[a];
            pot[o] = (OutT)((double)far_phi[a] + s.x);
            if (field) {
                field[3 * o] = (OutT)((double)far_E[a] + s.y);
                field[3 * o + 1] = (OutT)((double)far_E[npts + a] + s.z);
                field[3 * o + 2] = (OutT)((double)far_E[2 * npts + a] + s.w);
            }
        }
    }
}

// batched: one block per leaf of every system that has partial slots
template <typename OutT>
__global__ void __launch_bounds__(128)
k_b_p2p_combine(const BatchSys *__restrict__ S, const int32_t *__restrict__ off, int nsys) {
    const int s = batch_sys_of(off, nsys, blockIdx.x);
    const BatchSys &y = S[s];
    const int64_t t = blockIdx.x - off[s], nl = y.nleaf;
    const int p0 = y.poff[t], np = y.poff[t + 1] - p0;
    if (np == 0) return;
    const int nt = y.count[nl - 1 + t], bt = y.begin[nl - 1 + t];
    const int k = np / nt;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
        double4 a = y.partial[p0 + i];
        for (int j = 1; j < k; j++) {
            const double4 v = y.partial[p0 + j * nt + i];
            a.x += v.x;
            a.y += v.y;
            a.z += v.z;
            a.w += v.w;
        }
        const int64_t g = bt + i;
        const int64_t o = y.perm[g];
        ((OutT *)y.pot)[o] = (OutT)((double)y.far_phi[g] + a.x);
        if (y.field) {
            ((OutT *)y.field)[3 * o] = (OutT)((double)y.far_E[g] + a.y);
            ((OutT *)y.field)[3 * o + 1] = (OutT)((double)y.far_E[y.n + g] + a.z);
            ((OutT *)y.field)[3 * o + 2] = (OutT)((double)y.far_E[2 * y.n + g] + a.w);
        }
    }
}

}  // namespace

cudaError_t eval_p2p(Plan &P, void *pot, void *field, int dtype) {
    const unsigned grid = (unsigned)P.p2p_nunits;
    stage_mark(P, FMM_STAGE_P2P, 0);
    if (P.prec == FMM_PREC_MIXED) {
        cudaError_t e = mixed_p2p(P, pot, field, dtype);
        stage_mark(P, FMM_STAGE_P2P, 1);
        return e;
    }
    if (dtype == FMM_F64)
        FMM_LAUNCH(k_p2p_f64<double>, grid, kP2PThreads, 0, P.stream, P.B, P.n, P.x, P.y, P.z, P.q, P.begin,
                   P.count, P.ssrc[P.B], P.p2p_units, P.p2p_upart, P.p2p_nunits_dev, P.perm, P.far_phi, P.far_E,
                   P.p2p_partial, (double *)pot, (double *)field);
    else
        FMM_LAUNCH(k_p2p_f64<float>, grid, kP2PThreads, 0, P.stream, P.B, P.n, P.x, P.y, P.z, P.q, P.begin,
                   P.count, P.ssrc[P.B], P.p2p_units, P.p2p_upart, P.p2p_nunits_dev, P.perm, P.far_phi, P.far_E,
                   P.p2p_partial, (float *)pot, (float *)field);
    cudaError_t e = p2p_combine(P, pot, field, dtype);
    stage_mark(P, FMM_STAGE_P2P, 1);
    return e;
}

cudaError_t p2p_combine(Plan &P, void *pot, void *field, int dtype) {
    if (P.p2p_nparts == 0) return cudaGetLastError();
    const unsigned grid = (unsigned)std::min<int64_t>(P.nleaf, (int64_t)sm_count() * 8);
    const bool mixed = P.prec == FMM_PREC_MIXED;
    if (mixed && dtype == FMM_F64)
        FMM_LAUNCH((k_p2p_combine<double, float>), grid, 128, 0, P.stream, P.B, P.n, P.begin, P.count, P.p2p_poff,
                   P.p2p_partial, P.perm, P.far_phi_f, P.far_E_f, (double *)pot, (double *)field);
    else if (mixed)
        FMM_LAUNCH((k_p2p_combine<float, float>), grid, 128, 0, P.stream, P.B, P.n, P.begin, P.count, P.p2p_poff,
                   P.p2p_partial, P.perm, P.far_phi_f, P.far_E_f, (float *)pot, (float *)field);
    else if (dtype == FMM_F64)
        FMM_LAUNCH((k_p2p_combine<double, double>), grid, 128, 0, P.stream, P.B, P.n, P.begin, P.count,
                   P.p2p_poff, P.p2p_partial, P.perm, P.far_phi, P.far_E, (double *)pot, (double *)field);
    else
        FMM_LAUNCH((k_p2p_combine<float, double>), grid, 128, 0, P.stream, P.B, P.n, P.begin, P.count,
                   P.p2p_poff, P.p2p_partial, P.perm, P.far_phi, P.far_E, (float *)pot, (float *)field);
    return cudaGetLastError();
}

cudaError_t direct_run(const void *points, const void *charges, int64_t n, int dtype,
                       const int64_t *targets, int64_t nt, void *pot, void *field,
                       cudaStream_t s) {
    if (nt == 0) return cudaSuccess;
    if (dtype == FMM_F64)
        FMM_LAUNCH(k_direct<double>, (unsigned)nt, 256, 0, s, (const double *)points, (const double *)charges,
                                                      n, targets, (double *)pot, (double *)field);
    else
        FMM_LAUNCH(k_direct<float>, (unsigned)nt, 256, 0, s, (const float *)points, (const float *)charges, n,
                                                     targets, (float *)pot, (float *)field);
    return cudaGetLastError();
}

cudaError_t batch_combine(const BatchSys *S, const int32_t *off, int nsys, int64_t blocks, int dtype,
                          cudaStream_t st) {
    if (blocks == 0) return cudaGetLastError();
    if (dtype == FMM_F64)
        FMM_LAUNCH(k_b_p2p_combine<double>, (unsigned)blocks, 128, 0, st, S, off, nsys);
    else
        FMM_LAUNCH(k_b_p2p_combine<float>, (unsigned)blocks, 128, 0, st, S, off, nsys);
    return cudaGetLastError();
}

}  // namespace fmm
