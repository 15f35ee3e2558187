// Batched evaluation of many independent systems (Algorithm 1 per system,
// all systems at once).
//
// A batch of plans evaluated in mixed precision on binary levels with the
// single-precision M2L runs as one launch per stage over the work of every
// system: each block finds its system by a binary search in the stage's
// per-system block offsets (off[s] <= block < off[s + 1]). The stages whose
// kernels depend on the expansion order (M2M, M2L, L2L) run once per order
// present in the batch; the others read each system's order. A batch of one
// order is nine launches, whatever the number of systems:
//
//   prepare  charges into leaf order; zero the accumulated arrays
//   P2M      one block per leaf
//   M2M      one warp per leaf walking up (arrival counters), scaling each
//            completed multipole for the single-precision M2L
//   M2L      128-pair chunks of every system's weak pairs
//   L2L      one queue of 8-box chunks (bounded waits on the parent), each
//            box first taking its own unscaled M2L result
//   L2P      one block per leaf
//   P2P      the near-field work units of every system, heaviest first
//            (one launch per target tile size, 64 and 128)
//   combine  leaves whose strong list was cut into segments
//
// The work-unit lists of the systems are merged once, when the batch is
// made: units keep their weight bucket (a quarter octave of targets x
// sources) and the merged list is bucket-major, so the heaviest units of
// all systems start first.

#include <algorithm>
#include <cstring>
#include <vector>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int kPrepThreads = 256;
constexpr int64_t kPrepItems = 2048;  // per block and array

template <typename T>
__global__ void __launch_bounds__(kPrepThreads)
k_b_prepare(const BatchSys *__restrict__ S, const int32_t *__restrict__ off, int nsys, unsigned long long *next) {
    const int s = batch_sys_of(off, nsys, blockIdx.x);
    const BatchSys &y = S[s];
    if (blockIdx.x == 0 && threadIdx.x < kBatchMaxGroups) next[threadIdx.x] = 0ull;  // the L2L queues
    const int nc = ncoef(y.p);
    const int64_t nM = (y.nleaf - 1) * nc, nL = y.nbox * nc, end = std::max<int64_t>(y.n, nL);
    const int64_t stride = (int64_t)(off[s + 1] - off[s]) * blockDim.x;
    for (int64_t i = (blockIdx.x - off[s]) * (int64_t)blockDim.x + threadIdx.x; i < end; i += stride) {
        if (i < y.n) y.qf[i] = (float)((const T *)y.charges)[y.perm[i]];
        if (i < nM) y.M[i] = make_double2(0.0, 0.0);  // levels above the leaves (M2M adds into them)
        if (i < nL) y.Lh[i] = make_double2(0.0, 0.0);
        if (i < y.nbox) {
            y.arrive[i] = 0u;
            y.done[i] = 0;
        }
    }
}

// unit i of system s goes to dst[s][b] + (i - first unit of its bucket b)
__global__ void __launch_bounds__(256)
k_b_units_merge(const BatchSys *__restrict__ S, const int32_t *__restrict__ off, int nsys,
                const int32_t *__restrict__ dst, int4 *__restrict__ units, int32_t *__restrict__ upart,
                int32_t *__restrict__ usys) {
    const int s = batch_sys_of(off, nsys, blockIdx.x);
    const BatchSys &y = S[s];
    const int i = (int)(blockIdx.x - off[s]) * 256 + threadIdx.x;
    if (i >= y.ubstart[256]) return;
    int lo = 0, hi = 256;  // ubstart[lo] <= i < ubstart[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (y.ubstart[mid] <= i)
            lo = mid;
        else
            hi = mid;
    }
    const int64_t d = (int64_t)dst[(int64_t)s * 256 + lo] + (i - y.ubstart[lo]);
    units[d] = y.units[i];
    upart[d] = y.upart[i];
    usys[d] = s;
}

enum { kOffPrep, kOffLeaf, kOffComb, kOffMerge, kNumOff };
enum { kGrpM2M, kGrpM2L, kGrpL2L, kNumGrp };

size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

}  // namespace

bool batch_eligible(const Plan *const *plans, int n) {
    if (n < 1) return false;
    const Plan &A = *plans[0];
    bool seen[FMM_MAX_P + 1] = {};
    int groups = 0;
    for (int i = 0; i < n; i++) {
        const Plan &P = *plans[i];
        if (P.prec != FMM_PREC_MIXED || P.step != 1 || !P.Mf || P.m2l_tc || !P.f32_tab || !P.box_geo || !P.box_cf) return false;
        if (P.dtype != A.dtype || P.device != A.device) return false;
        if (!seen[P.p]) seen[P.p] = true, groups++;
    }
    return groups <= kBatchMaxGroups;
}

void batch_release(BatchRun &R) {
    if (R.mem) cudaFree(R.mem);
    R = BatchRun{};
}

cudaError_t batch_setup(const Plan *const *plans, int n, const void *const *charges, void *const *pot,
                        void *const *field, BatchRun &R, cudaStream_t st) {
    R = BatchRun{};
    // the orders present, ascending; group of each system
    int gof[FMM_MAX_P + 1];
    for (int q = 0; q <= FMM_MAX_P; q++) gof[q] = -1;
    for (int i = 0; i < n; i++) gof[plans[i]->p] = 0;
    int G = 0;
    for (int q = 0; q <= FMM_MAX_P; q++)
        if (gof[q] == 0) {
            gof[q] = G;
            R.grp[G].p = q;
            G++;
        }
    R.ngroups = G;
    R.pmax = R.grp[G - 1].p;
    // per-system block counts of each stage, and the systems' weight buckets
    std::vector<std::vector<int64_t>> cnt(kNumOff, std::vector<int64_t>(n));
    std::vector<std::vector<std::vector<int64_t>>> gcnt(
        G, std::vector<std::vector<int64_t>>(kNumGrp, std::vector<int64_t>(n, 0)));
    std::vector<int32_t> bst((size_t)n * 257);
    std::vector<BatchSys> hs(n);
    for (int i = 0; i < n; i++) {
        const Plan &P = *plans[i];
        cudaError_t e = cudaMemcpy(&bst[(size_t)i * 257], P.p2p_bstart, 257 * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return e;
        BatchSys &y = hs[i];
        std::memset(&y, 0, sizeof(y));
        y.B = P.B;
        y.lw = first_weak_level_of(P);
        y.dtype = P.dtype;
        y.p = P.p;
        y.n = P.n;
        y.nbox = P.nbox;
        y.nleaf = P.nleaf;
        y.npairs = total_weak(P);
        y.perm = P.perm;
        y.begin = P.begin;
        y.count = P.count;
        y.ssrc = P.ssrc[P.B];
        y.poff = P.p2p_poff;
        y.centre = P.centre;
        y.radius = P.radius;
        y.hl = P.hl;
        y.qf = P.qf;
        y.far_phi = P.far_phi_f;
        y.far_E = P.far_E_f;
        y.lgeo = P.lgeo;
        y.M = P.M;
        y.L = P.L;
        y.Lh = P.Lh;
        y.Mf = P.Mf;
        y.arrive = P.m2m_arrive;
        y.done = P.l2l_done;
        y.err = P.d_err;
        y.charges = charges[i];
        y.pot = pot[i];
        y.field = field ? field[i] : nullptr;
        y.partial = P.p2p_partial;
        y.units = P.p2p_units;
        y.upart = P.p2p_upart;
        y.ubstart = P.p2p_bstart;
        y.box_geo = P.box_geo;
        y.box_cf = P.box_cf;
        y.pt = pair_table(P);
        cnt[kOffPrep][i] =
            std::max<int64_t>(1, (std::max<int64_t>(P.n, P.nbox * P.nc) + kPrepItems - 1) / kPrepItems);
        cnt[kOffLeaf][i] = P.nleaf;
        cnt[kOffComb][i] = P.p2p_nparts ? P.nleaf : 0;
        cnt[kOffMerge][i] = (P.p2p_nunits + 255) / 256;
        const int g = gof[P.p];
        gcnt[g][kGrpM2M][i] = (P.nleaf + kWarpChildMax - 1) / kWarpChildMax;
        gcnt[g][kGrpM2L][i] = (y.npairs + 127) / 128;
        gcnt[g][kGrpL2L][i] = (P.nbox + 7) / 8;
        if (!R.grp[g].tab) {
            R.grp[g].tab = P.m2l_tab;
            R.grp[g].tab_df = P.m2l_tab_df;
            R.grp[g].ftab = P.f32_tab;
        }
    }
    // block offsets; every total must fit the int32 tables
    std::vector<std::vector<int32_t>> off;
    auto offsets = [&](const std::vector<int64_t> &c, int64_t &total) -> bool {
        std::vector<int32_t> o(n + 1);
        int64_t t = 0;
        for (int i = 0; i < n; i++) {
            o[i] = (int32_t)t;
            t += c[i];
            if (t > 0x7fffffffLL) return false;
        }
        o[n] = (int32_t)t;
        total = t;
        off.push_back(std::move(o));
        return true;
    };
    for (int k = 0; k < kNumOff; k++)
        if (!offsets(cnt[k], R.blocks[k])) return cudaErrorInvalidValue;
    for (int g = 0; g < G; g++)
        for (int k = 0; k < kNumGrp; k++)
            if (!offsets(gcnt[g][k], R.grp[g].blocks[k])) return cudaErrorInvalidValue;
    const int ntab = (int)off.size();  // kNumOff + G * kNumGrp
    // merged unit list: tile-64 systems first, then tile-128; within each,
    // bucket-major, then system order, then each system's own order
    std::vector<int32_t> dst((size_t)n * 256, 0);
    int64_t base = 0;
    for (int cls = 0; cls < 2; cls++) {
        const int tile = cls == 0 ? kP2PTileSmall : kP2PTile;
        const int64_t start = base;
        for (int b = 0; b < 256; b++)
            for (int i = 0; i < n; i++) {
                if (plans[i]->p2p_tile != tile) continue;
                const int32_t *bs = &bst[(size_t)i * 257];
                dst[(size_t)i * 256 + b] = (int32_t)base;
                base += bs[b + 1] - bs[b];
                if (base > 0x7fffffffLL) return cudaErrorInvalidValue;
            }
        R.nunits[cls] = base - start;
    }
    const int64_t nu = base;
    // one device block: descriptors, offsets, destinations, merged units, queue counters
    size_t o = 0;
    const size_t oS = o;
    o += align16(sizeof(BatchSys) * n);
    const size_t oOff = o;
    o += align16((size_t)ntab * (n + 1) * 4);
    const size_t oDst = o;
    o += align16(dst.size() * 4);
    const size_t hostBytes = o;
    const size_t oUnits = o;
    o += align16((size_t)std::max<int64_t>(nu, 1) * sizeof(int4));
    const size_t oUpart = o;
    o += align16((size_t)std::max<int64_t>(nu, 1) * 4);
    const size_t oUsys = o;
    o += align16((size_t)std::max<int64_t>(nu, 1) * 4);
    const size_t oNext = o;
    o += align16(kBatchMaxGroups * 8);
    std::vector<char> host(hostBytes, 0);
    std::memcpy(host.data() + oS, hs.data(), sizeof(BatchSys) * n);
    for (int k = 0; k < ntab; k++) std::memcpy(host.data() + oOff + (size_t)k * (n + 1) * 4, off[k].data(), (n + 1) * 4);
    std::memcpy(host.data() + oDst, dst.data(), dst.size() * 4);
    cudaError_t e = cudaMalloc(&R.mem, o);
    if (e != cudaSuccess) {
        R.mem = nullptr;
        return e;
    }
    char *m = (char *)R.mem;
    R.nsys = n;
    R.dtype = plans[0]->dtype;
    R.S = (BatchSys *)(m + oS);
    int32_t *ot = (int32_t *)(m + oOff);
    for (int k = 0; k < kNumOff; k++) R.off[k] = ot + (size_t)k * (n + 1);
    for (int g = 0; g < G; g++)
        for (int k = 0; k < kNumGrp; k++) R.grp[g].off[k] = ot + (size_t)(kNumOff + g * kNumGrp + k) * (n + 1);
    R.units = (int4 *)(m + oUnits);
    R.upart = (int32_t *)(m + oUpart);
    R.usys = (int32_t *)(m + oUsys);
    R.next = (unsigned long long *)(m + oNext);
    e = cudaMemcpyAsync(m, host.data(), hostBytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && R.blocks[kOffMerge] > 0)
        FMM_LAUNCH(k_b_units_merge, (unsigned)R.blocks[kOffMerge], 256, 0, st, R.S, R.off[kOffMerge], n,
                   (const int32_t *)(m + oDst), R.units, R.upart, R.usys);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = batch_smem_limits(R.pmax);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host tables go out of scope
    if (e != cudaSuccess) batch_release(R);
    return e;
}

// one batched evaluation, on `st`: six launches plus three per order present
cudaError_t batch_enqueue(const BatchRun &R, cudaStream_t st) {
    const int n = R.nsys;
    if (R.dtype == FMM_F64)
        FMM_LAUNCH(k_b_prepare<double>, (unsigned)R.blocks[kOffPrep], kPrepThreads, 0, st, R.S, R.off[kOffPrep], n,
                   R.next);
    else
        FMM_LAUNCH(k_b_prepare<float>, (unsigned)R.blocks[kOffPrep], kPrepThreads, 0, st, R.S, R.off[kOffPrep], n,
                   R.next);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = batch_p2m(R.S, R.off[kOffLeaf], n, R.blocks[kOffLeaf], R.pmax, st);
    for (int g = 0; g < R.ngroups && e == cudaSuccess; g++) {
        const BatchGroup &G = R.grp[g];
        e = batch_m2m_up(R.S, G.off[kGrpM2M], n, G.blocks[kGrpM2M], G.p, G.tab_df, st);
    }
    for (int g = 0; g < R.ngroups && e == cudaSuccess; g++) {
        const BatchGroup &G = R.grp[g];
        e = batch_m2l(R.S, G.off[kGrpM2L], n, G.blocks[kGrpM2L], G.p, G.ftab, st);
    }
    for (int g = 0; g < R.ngroups && e == cudaSuccess; g++) {
        const BatchGroup &G = R.grp[g];
        e = batch_l2l_down(R.S, G.off[kGrpL2L], n, G.blocks[kGrpL2L], G.p, G.tab, G.tab_df, R.next + g, st);
    }
    if (e == cudaSuccess) e = batch_l2p(R.S, R.off[kOffLeaf], n, R.blocks[kOffLeaf], R.pmax, st);
    if (e == cudaSuccess) e = batch_p2p(R.S, R.units, R.usys, R.upart, R.nunits[0], kP2PTileSmall, R.dtype, st);
    if (e == cudaSuccess)
        e = batch_p2p(R.S, R.units + R.nunits[0], R.usys + R.nunits[0], R.upart + R.nunits[0], R.nunits[1], kP2PTile,
                      R.dtype, st);
    if (e == cudaSuccess) e = batch_combine(R.S, R.off[kOffComb], n, R.blocks[kOffComb], R.dtype, st);
    return e;
}

}  // namespace fmm
