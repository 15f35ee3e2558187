// Internal declarations of the GB300 FMM library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <utility>
#include <vector>

#include "fmm.h"

namespace fmm {

// targets per near-field work unit (one CTA, one target per thread): at most
// kP2PTile; the mixed form takes kP2PTileSmall when the leaves hold 64 points
// or fewer on average, so that a unit's threads are not half idle
constexpr int kP2PTile = 128;
constexpr int kP2PTileSmall = 64;
// sources per near-field work unit at most (about): a target leaf whose
// strong list holds more is cut into segments, each its own unit
constexpr int kP2PSegSources = 1 << 16;

// ---------------------------------------------------------------------------
// Plan: everything lives in device memory owned by the plan.
// ---------------------------------------------------------------------------
// Bump allocator over a few large blocks from the caller's allocator: a plan
// makes a handful of allocator calls instead of one per buffer.
struct Arena {
    std::vector<std::pair<void *, size_t>> blocks;
    char *cur = nullptr;
    size_t left = 0, hint = 0;
};

// weak pairs of every level, concatenated (levels lmin..lmax); passed by value
struct PairTable {
    const int32_t *tgt[FMM_MAX_LEVELS + 1];
    const int32_t *src[FMM_MAX_LEVELS + 1];
    long long off[FMM_MAX_LEVELS + 2];
    int lmin, lmax;
};

// One system of a batched evaluation as the batched stage kernels read it
// (an array of these lives on the device): the plan's arrays, its sizes,
// its first level with weak pairs, its caller's charges and outputs.
// warps (one child box each) per block of the M2M/L2L kernels
constexpr int kWarpChildMax = 8;

struct BatchSys {
    int B, lw, dtype, p;
    int64_t n, nbox, nleaf, npairs;
    const int32_t *perm, *begin, *count, *ssrc, *poff;
    const double *centre, *radius;
    const float *hl;
    float *qf, *far_phi, *far_E;
    const float4 *lgeo;
    double2 *M, *L, *Lh;
    float2 *Mf;
    unsigned *arrive;
    int *done, *err;
    const void *charges;
    void *pot, *field;
    double4 *partial;
    const void *box_geo;           // per box: geometry of the translation to / from its parent
    const float4 *box_cf;          // per box: centre hi (xyz) + radius, centre lo
    const int4 *units;             // near-field work units, heaviest bucket first
    const int32_t *upart, *ubstart;
    PairTable pt;
};

// (ah + al) - (bh + bl) in float from the split values: TwoSum of the hi
// parts, then the error and the lo parts
__device__ __forceinline__ float offset_f(float ah, float bh, float al, float bl) {
    const float d = __fsub_rn(ah, bh);
    const float bb = __fsub_rn(d, ah);
    const float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(d, bb)), __fsub_rn(-bh, bb));
    return __fadd_rn(d, __fadd_rn(e, __fsub_rn(al, bl)));
}

// 2^k as a double, for |k| <= 1022 (exact; integer operations only)
__device__ __forceinline__ double pow2i(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }

// Block b of a batched launch belongs to system s with off[s] <= b < off[s+1].
__device__ __forceinline__ int batch_sys_of(const int32_t *__restrict__ off, int nsys, int64_t b) {
    int lo = 0, hi = nsys;  // off[lo] <= b < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= b)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// A given root cell (FMM_FLAG_ROOT_CELL), passed to the root kernel by value.
struct RootCell {
    double lo[3] = {0.0, 0.0, 0.0}, hi[3] = {0.0, 0.0, 0.0};
    int given = 0;
};

struct Plan {
    int64_t n = 0;
    int B = 0, p = 0, nc = 0, prec = 0, dtype = 0, device = 0;
    double theta = 0.0;
    double eta = 1.0;  // adaptivity of the splits (Sec. 2.1.2); 1: median splits
    int step = 1;      // bisections per expansion level (3: octree levels)
    int64_t nbox = 0, nleaf = 0;
    cudaStream_t stream = nullptr;
    fmm_allocator alloc{};
    bool has_alloc = false;

    // points in leaf order (structure of arrays) and slot -> original index
    double *x = nullptr, *y = nullptr, *z = nullptr;
    int32_t *perm = nullptr;
    // boxes in heap order
    int32_t *begin = nullptr;   // first leaf-order slot of each box
    int32_t *count = nullptr;   // points per box
    double *lo = nullptr, *hi = nullptr, *centre = nullptr;   // nbox x 3
    double *radius = nullptr, *plane = nullptr;               // nbox
    int32_t *axis = nullptr;                                  // nbox
    // FMM_FLAG_TIGHT: centre/radius from each box's points; their bounding
    // boxes (nbox x 3 each) live until fmm_plan returns
    bool tight = false;
    double *tlo = nullptr, *thi = nullptr;
    RootCell root;  // FMM_FLAG_ROOT_CELL
    // one rank's part of a system split over several devices: every level's
    // multipoles are formed; local expansions (nbox x nc) and near-field
    // terms (4 per point, leaf order) from the other ranks are added during
    // the downward pass
    bool full_upward = false, ext_active = false;
    double2 *L_ext = nullptr;
    double *near_ext = nullptr;
    // connectivity: CSR per level over the 2^l target boxes of level l
    int32_t *wptr[FMM_MAX_LEVELS + 1] = {}, *wsrc[FMM_MAX_LEVELS + 1] = {};
    int32_t *sptr[FMM_MAX_LEVELS + 1] = {}, *ssrc[FMM_MAX_LEVELS + 1] = {};
    int32_t *wrow[FMM_MAX_LEVELS + 1] = {};  // target of every weak pair (flat M2L)
    int64_t nweak[FMM_MAX_LEVELS + 1] = {}, nstrong[FMM_MAX_LEVELS + 1] = {};
    unsigned long long *p2p_work_dev = nullptr;  // exact near-field pair count (device)
    // near-field work units (target leaf, first target, strong-list segment
    // [begin, end)), heaviest first; their number on the device and on the
    // host; per unit its partial-sum slot base (-1: the leaf is not split);
    // per leaf the offset of its k * n_t partial slots (scan); the slots
    int4 *p2p_units = nullptr;
    int32_t *p2p_upart = nullptr;
    const int32_t *p2p_nunits_dev = nullptr;
    int64_t p2p_nunits = 0;
    int32_t *p2p_poff = nullptr;
    int64_t p2p_nparts = 0;
    double4 *p2p_partial = nullptr;
    int p2p_tile = kP2PTile;  // targets per work unit (kP2PTile or kP2PTileSmall)
    int32_t *p2p_bstart = nullptr;  // first unit of each of the 256 weight buckets; [256] = units
    bool capacity_exceeded = false;
    // M2L rotation tables (D = d(pi/2) quadrants, axial coefficients, F_nm)
    double *m2l_tab = nullptr;
    // mixed form: the same tables as double-float pairs (hi, lo floats), and
    // per box the geometry of its translation from / to its parent
    float2 *m2l_tab_df = nullptr;
    void *box_geo = nullptr;
    // per box its centre split hi + lo in float and its radius (hi.w): the
    // theta-test's pre-test and the single-precision M2L form offsets from
    // them without double arithmetic
    float4 *box_cf = nullptr;
    unsigned *m2m_arrive = nullptr;         // one-launch upward pass: arrivals per parent
    int *l2l_done = nullptr;                // one-launch downward pass: box finished
    unsigned long long *l2l_next = nullptr; // one-launch downward pass: next box to take
    int m2l_ntab = 0, m2l_threads = 0;
    size_t m2l_smem = 0;
    // mixed precision: leaf offsets hi|lo (6n floats), float charges and far
    // field, radius-scaled float multipoles for the single-precision M2L
    float *hl = nullptr, *qf = nullptr, *far_phi_f = nullptr, *far_E_f = nullptr;
    float4 *lgeo = nullptr;  // per leaf: centre hi (xyz, radius) | centre lo | half extents
    bool m2l_tc = false;     // mixed form: M2L on the tensor cores (else the SIMT float kernel)
    bool tc_m2l_opt = false; // FMM_FLAG_TC_M2L requested
    void *tc_tab = nullptr;  // tensor-core M2L tables (per device and order, not owned)
    void *f32_tab = nullptr;  // packed coefficient-pair tables of the float M2L (plan-owned)
    int tc_ctas = 0;
    float2 *Mf = nullptr;
    double2 *Lh = nullptr;  // r^k-scaled locals accumulated by the float M2L
    // evaluation scratch
    double *q = nullptr;                 // charges in leaf order
    double2 *M = nullptr, *L = nullptr;  // nbox x nc
    double *far_phi = nullptr;           // n, leaf order
    double *far_E = nullptr;             // 3n, leaf order (SoA: x | y | z)
    // staging for host arguments
    void *stage = nullptr;
    size_t stage_bytes = 0;
    int *d_err = nullptr;                // device error word
    // per-stage device timing (FMM_FLAG_PROFILE)
    bool profile = false;
    cudaEvent_t ev[FMM_NSTAGES][2] = {};
    // plan-lifetime buffers (released by fmm_destroy) and fmm_plan temporaries
    // (released when fmm_plan returns)
    Arena persist, scratch;
};

// Allocation through the plan's allocator (or stream-ordered cudaMallocAsync).
// palloc: owned by the plan until fmm_destroy; dalloc: temporary of fmm_plan,
// released in bulk when fmm_plan returns (dfree is then a no-op marker).
void *dalloc(Plan &P, size_t bytes);
void dfree(Plan &P, void *ptr, size_t bytes);
void *palloc(Plan &P, size_t bytes);
void arena_release(Plan &P, Arena &A);

// cudaError_t -> fmm_status; records the code for fmm_last_cuda_error().
int cuda_status(cudaError_t e);
// Where a caller's pointer lives: 1 = device memory of the current device
// (or managed memory), 0 = host memory (pageable, pinned or unregistered),
// -1 = device memory of another device (rejected: the kernels run on the
// current device and cannot dereference it).
int ptr_kind(const void *p);

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount,
// read once per device); grids are sized in multiples of it.
int sm_count();

// Kernel launches made by the library (fmm_kernel_launches).
extern std::atomic<long long> g_launches;
#define FMM_LAUNCH(kernel, grid, block, smem, stream, ...)          \
    do {                                                            \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__); \
        ::fmm::g_launches.fetch_add(1, std::memory_order_relaxed);  \
    } while (0)

// Stage timing marks (no-ops unless the plan profiles).
inline void stage_mark(Plan &P, int stage, int edge) {
    if (P.profile) cudaEventRecord(P.ev[stage][edge], P.stream);
}

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__host__ __device__ inline int tri(int n, int m) { return n * (n + 1) / 2 + m; }
__host__ __device__ inline int ncoef(int p) { return (p + 1) * (p + 2) / 2; }
// row stride (coefficients) of the float multipoles Mf: even, so that
// coefficient pairs (2i, 2i+1) are 16-byte aligned
__host__ __device__ inline int mf_stride(int p) { return (ncoef(p) + 1) & ~1; }

// Order-preserving map from doubles to unsigned 64-bit keys (no NaN; -0 was
// canonicalised to +0 on input).
__device__ __forceinline__ uint64_t dkey(double v) {
    uint64_t u = (uint64_t)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(uint64_t k) {
    uint64_t u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)u);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
    return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) {
    return make_double2(a.x * s, a.y * s);
}

// Coefficient C_n^m of a real-source expansion stored for m >= 0:
// C_n^{-m} = (-1)^m conj(C_n^m); zero outside |m| <= n.
__device__ __forceinline__ double2 coef_at(const double2 *C, int n, int m) {
    if (n < 0 || m > n || -m > n) return make_double2(0.0, 0.0);
    if (m >= 0) return C[tri(n, m)];
    double2 c = C[tri(n, -m)];
    return ((-m) & 1) ? make_double2(-c.x, c.y) : make_double2(c.x, -c.y);
}

// ---------------------------------------------------------------------------
// Host-side launchers (each in its own translation unit)
// ---------------------------------------------------------------------------
cudaError_t tree_build(Plan &P, const void *points_dev, int dtype);
cudaError_t tight_geometry(Plan &P);
cudaError_t lists_build(Plan &P);
cudaError_t direct_run(const void *points, const void *charges, int64_t n, int dtype,
                       const int64_t *targets, int64_t nt, void *pot, void *field,
                       cudaStream_t s);
cudaError_t m2l_setup(Plan &P);
cudaError_t theta_pairs(double theta, int64_t n, const double *ca, const double *ra, const double *cb,
                        const double *rb, uint8_t *weak, cudaStream_t st);
cudaError_t eval_upward(Plan &P, const void *charges, int dtype);
cudaError_t eval_expansions(Plan &P, const void *charges, int dtype);
cudaError_t eval_p2p(Plan &P, void *pot, void *field, int dtype);
cudaError_t eval_downward(Plan &P);
cudaError_t add_external_locals(Plan &P);
cudaError_t add_external_near(Plan &P);
// batched stages: every system of a batch (same order, mixed form, binary
// levels) in one launch per stage; `off` holds per-system block (or chunk)
// offsets, off[nsys] = the total
cudaError_t batch_p2m(const BatchSys *S, const int32_t *off, int nsys, int64_t blocks, int pmax, cudaStream_t st);
cudaError_t batch_m2m_up(const BatchSys *S, const int32_t *off, int nsys, int64_t blocks, int p,
                         const float2 *tab_df, cudaStream_t st);
cudaError_t batch_m2l(const BatchSys *S, const int32_t *off, int nsys, int64_t nchunks, int p, const void *tab,
                      cudaStream_t st);
cudaError_t batch_l2l_down(const BatchSys *S, const int32_t *off, int nsys, int64_t nchunks, int p,
                           const double *tab, const float2 *tab_df, unsigned long long *next, cudaStream_t st);
cudaError_t batch_l2p(const BatchSys *S, const int32_t *off, int nsys, int64_t blocks, int pmax, cudaStream_t st);
cudaError_t batch_p2p(const BatchSys *S, const int4 *units, const int32_t *usys, const int32_t *upart, int64_t n,
                      int tile, int dtype, cudaStream_t st);
cudaError_t batch_combine(const BatchSys *S, const int32_t *off, int nsys, int64_t blocks, int dtype,
                          cudaStream_t st);
cudaError_t batch_smem_limits(int p);

// a batch's device tables (batch.cu): descriptors, per-stage block offsets
// (the order-dependent stages per group of systems of one order), the merged
// near-field units, the L2L queue counters; one allocation
constexpr int kBatchMaxGroups = 8;
struct BatchGroup {
    int p = 0;
    int32_t *off[3] = {};    // M2M blocks, M2L chunks, L2L chunks (other orders: none)
    int64_t blocks[3] = {};
    const double *tab = nullptr;
    const float2 *tab_df = nullptr;
    const void *ftab = nullptr;
};
struct BatchRun {
    void *mem = nullptr;
    int nsys = 0, pmax = 0, dtype = 0, ngroups = 0;
    BatchSys *S = nullptr;
    int32_t *off[4] = {};    // prepare, leaves (P2M, L2P), combine, unit merge
    int64_t blocks[4] = {};
    BatchGroup grp[kBatchMaxGroups];
    int4 *units = nullptr;
    int32_t *upart = nullptr, *usys = nullptr;
    int64_t nunits[2] = {0, 0};  // tile 64, tile 128
    unsigned long long *next = nullptr;  // one L2L queue counter per group
};
bool batch_eligible(const Plan *const *plans, int n);
cudaError_t batch_setup(const Plan *const *plans, int n, const void *const *charges, void *const *pot,
                        void *const *field, BatchRun &R, cudaStream_t st);
cudaError_t batch_enqueue(const BatchRun &R, cudaStream_t st);
void batch_release(BatchRun &R);
int first_weak_level_of(const Plan &P);
// P.box_cf from the final box geometry (the list build makes it)
void box_centres_f(Plan &P);
PairTable pair_table(const Plan &P);
int64_t total_weak(const Plan &P);

// FP64 M2L from multipoles outside the plan into L_ext: n pairs (target box
// `tgt[i]` of `level`, source i with multipole M[i] about centre[i])
cudaError_t m2l_external(Plan &P, int level, int64_t n, const int32_t *tgt, const double2 *M,
                         const double *centre);
cudaError_t m2l_all(Plan &P);
void m2m_level(Plan &P, int level);
void l2l_level(Plan &P, int level);
void m2m_up(Plan &P, int stop);
void l2l_down(Plan &P, int lw);
bool m2l_f32_supported(int p);
// Raises a kernel's dynamic shared-memory limit to the device's opt-in
// maximum (never lowers it): plans of different orders share the kernels,
// and a per-plan value would let one plan shrink another's limit.
cudaError_t allow_max_smem(const void *func, size_t need);
bool m2l_tc_supported(int p);
cudaError_t m2l_tc_setup(Plan &P);
cudaError_t m2l_tc_launch(Plan &P);
cudaError_t m2l_f32_setup(Plan &P);
cudaError_t m2l_f32_all(Plan &P);
cudaError_t mixed_setup(Plan &P);
cudaError_t mixed_p2m(Plan &P, const void *charges, int dtype);
cudaError_t mixed_l2p(Plan &P);
cudaError_t mixed_p2p(Plan &P, void *pot, void *field, int dtype);
// adds the partial near-field sums of split leaves in segment order, plus the
// far field, and writes those leaves' outputs in input order
cudaError_t p2p_combine(Plan &P, void *pot, void *field, int dtype);
// device-wide exclusive scan of int32 counts (n + 1 outputs, last = total)
cudaError_t scan_exclusive(Plan &P, const int32_t *in, int32_t *out, int64_t n);

}  // namespace fmm

// The handle behind fmm_plan_t.
struct fmm_plan_s {
    fmm::Plan P;
};
