// C ABI of the GB300 FMM library: argument checking, memory ownership,
// host/device staging and the stage order of Algorithm 1 (Tree in fmm_plan;
// P2M, M2M, M2L, L2L, L2P, P2P in fmm_eval).

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fmm_internal.cuh"

namespace fmm {

std::atomic<long long> g_launches{0};

namespace {
thread_local int g_last_cuda = 0;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return FMM_OK;
    g_last_cuda = (int)e;
    if (e == cudaErrorMemoryAllocation) return FMM_ENOMEM;
    return FMM_ECUDA;
}

int ptr_kind(const void *p) {
    if (!p) return 0;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeManaged) return 1;
    if (a.type != cudaMemoryTypeDevice) return 0;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return a.device == dev ? 1 : -1;
}

int sm_count() {
    static std::atomic<int> cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 148;
    }
    int v = cached[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
        cudaGetLastError();
        return 148;
    }
    cached[dev].store(v, std::memory_order_relaxed);
    return v;
}

namespace {

// Without a caller's allocator, plan memory comes from a stream-ordered pool
// of the library's own per device that keeps freed memory for the next plan
// (the device's default pool returns it at every synchronisation, so each
// plan would map its ~100 bytes per point anew); fmm_pool_trim releases it.
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};

cudaMemPool_t library_pool(int dev) {
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}

void *raw_alloc(Plan &P, size_t bytes) {
    if (P.has_alloc) return P.alloc.alloc(bytes, P.alloc.ctx, (void *)P.stream);
    int dev = 0;
    void *p = nullptr;
    cudaMemPool_t pool = cudaGetDevice(&dev) == cudaSuccess ? library_pool(dev) : nullptr;
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, P.stream)
                               : cudaMallocAsync(&p, bytes, P.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void raw_free(Plan &P, void *ptr, size_t bytes) {
    if (P.has_alloc)
        P.alloc.free(ptr, bytes, P.alloc.ctx, (void *)P.stream);
    else
        cudaFreeAsync(ptr, P.stream);
}

void *arena_alloc(Plan &P, Arena &A, size_t bytes) {
    bytes = (std::max<size_t>(bytes, 1) + 255) & ~(size_t)255;
    if (bytes > A.left) {
        const size_t bs = std::max(bytes, std::max<size_t>(A.hint, 1 << 20));
        void *p = raw_alloc(P, bs);
        if (!p) return nullptr;
        A.blocks.push_back({p, bs});
        A.cur = (char *)p;
        A.left = bs;
        A.hint = std::max<size_t>(A.hint / 2, 1 << 20);  // later blocks: smaller
    }
    void *r = A.cur;
    A.cur += bytes;
    A.left -= bytes;
    return r;
}

}  // namespace

void arena_release(Plan &P, Arena &A) {
    for (auto it = A.blocks.rbegin(); it != A.blocks.rend(); ++it) raw_free(P, it->first, it->second);
    A.blocks.clear();
    A.cur = nullptr;
    A.left = 0;
}

void *dalloc(Plan &P, size_t bytes) { return arena_alloc(P, P.scratch, bytes); }
void dfree(Plan &, void *, size_t) {}
void *palloc(Plan &P, size_t bytes) { return arena_alloc(P, P.persist, bytes); }

}  // namespace fmm

using fmm::Plan;
using fmm::cuda_status;

struct fmm_batch_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    cudaStream_t own = nullptr;
    fmm::BatchRun run;  // batched stages (one launch per stage over all systems)
    bool fused = false;
    int64_t kernels = 0;  // kernel nodes of the graph
};

namespace {

bool is_device_ptr(const void *p) { return fmm::ptr_kind(p) == 1; }

void release(Plan &P) {
    for (int s = 0; s < FMM_NSTAGES; s++)
        for (int e = 0; e < 2; e++)
            if (P.ev[s][e]) cudaEventDestroy(P.ev[s][e]);
    fmm::arena_release(P, P.scratch);
    fmm::arena_release(P, P.persist);
    cudaStreamSynchronize(P.stream);
    cudaGetLastError();
}

size_t dsize(int dtype) { return dtype == FMM_F64 ? 8 : 4; }

}  // namespace

extern "C" {

int fmm_stage_times(fmm_plan_t plan, double *ms) {
    if (!plan || !ms || !plan->P.profile) return FMM_EINVAL;
    Plan &P = plan->P;
    cudaError_t e = cudaStreamSynchronize(P.stream);
    for (int s = 0; s < FMM_NSTAGES && e == cudaSuccess; s++) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, P.ev[s][0], P.ev[s][1]);
        ms[s] = t;
    }
    return cuda_status(e);
}

int64_t fmm_kernel_launches(void) { return (int64_t)fmm::g_launches.load(); }

const char *fmm_strerror(int status) {
    switch (status) {
        case FMM_OK: return "success";
        case FMM_EINVAL: return "invalid argument";
        case FMM_ENOMEM: return "device allocation failed";
        case FMM_ENONFINITE: return "non-finite point coordinate";
        case FMM_ECAPACITY: return "interaction list exceeds 2^31-1 entries";
        case FMM_ETIMEDOUT: return "bounded device wait timed out";
        case FMM_ECUDA: return "CUDA runtime error";
        case FMM_EINTERNAL: return "internal consistency check of the tree build failed";
        default: return "unknown status";
    }
}

int fmm_last_cuda_error(void) { return fmm::g_last_cuda; }

int fmm_pool_trim(int device) {
    if (device < 0 || device >= 64) return FMM_EINVAL;
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(fmm::g_pool_mu);
        pool = fmm::g_pool[device];
    }
    if (!pool) return FMM_OK;
    return cuda_status(cudaMemPoolTrimTo(pool, 0));
}

int fmm_plan(const void *points, int64_t n, int dtype, const fmm_opts *opts,
             const fmm_allocator *alloc, void *stream, fmm_plan_t *out) {
    if (out) *out = nullptr;
    if (!out || !points || !opts) return FMM_EINVAL;
    if (n < 1 || n > 0x7fffffffLL) return FMM_EINVAL;
    if (dtype != FMM_F64 && dtype != FMM_F32) return FMM_EINVAL;
    if (opts->levels < 0 || opts->levels > FMM_MAX_LEVELS) return FMM_EINVAL;
    if (opts->p < 0 || opts->p > FMM_MAX_P) return FMM_EINVAL;
    if (!(opts->theta >= 0.0 && opts->theta < 1.0)) return FMM_EINVAL;
    if (opts->prec != FMM_PREC_FP64 && opts->prec != FMM_PREC_MIXED) return FMM_EINVAL;
    if (opts->flags & ~(FMM_FLAG_PROFILE | FMM_FLAG_ETA | FMM_FLAG_TC_M2L | FMM_FLAG_TIGHT | FMM_FLAG_ROOT_CELL))
        return FMM_EINVAL;
    if (opts->flags & FMM_FLAG_ROOT_CELL)
        for (int a = 0; a < 3; a++)
            if (!(std::isfinite(opts->root_lo[a]) && std::isfinite(opts->root_hi[a]) &&
                  opts->root_lo[a] <= opts->root_hi[a]))
                return FMM_EINVAL;
    if ((opts->flags & FMM_FLAG_ETA) && !(opts->eta >= 0.0 && opts->eta <= 1.0)) return FMM_EINVAL;
    const int step = opts->bisections_per_level == 0 ? 1 : opts->bisections_per_level;
    if (step < 1 || step > 3 || opts->levels % step != 0) return FMM_EINVAL;
    if (alloc && (!alloc->alloc || !alloc->free)) return FMM_EINVAL;
    if (fmm::ptr_kind(points) < 0) return FMM_EINVAL;

    fmm_plan_s *H = new (std::nothrow) fmm_plan_s();
    if (!H) return FMM_ENOMEM;
    Plan &P = H->P;
    P.n = n;
    P.B = opts->levels;
    P.p = opts->p;
    P.nc = fmm::ncoef(P.p);
    P.theta = opts->theta;
    P.eta = (opts->flags & FMM_FLAG_ETA) ? opts->eta : 1.0;
    P.step = step;
    P.prec = opts->prec;
    P.dtype = dtype;
    P.nbox = ((int64_t)2 << P.B) - 1;
    P.nleaf = (int64_t)1 << P.B;
    P.stream = (cudaStream_t)stream;
    if (alloc) {
        P.alloc = *alloc;
        P.has_alloc = true;
    }
    cudaGetDevice(&P.device);
    P.profile = (opts->flags & FMM_FLAG_PROFILE) != 0;
    P.tc_m2l_opt = (opts->flags & FMM_FLAG_TC_M2L) != 0;
    P.tight = (opts->flags & FMM_FLAG_TIGHT) != 0;
    if (opts->flags & FMM_FLAG_ROOT_CELL) {
        P.root.given = 1;
        for (int a = 0; a < 3; a++) {
            P.root.lo[a] = opts->root_lo[a];
            P.root.hi[a] = opts->root_hi[a];
        }
    }

    auto fail = [&](int status) {
        release(P);
        delete H;
        return status;
    };

    // arena sizes: points, boxes, expansions and a guess for the lists
    P.persist.hint = (size_t)n * 96 + (size_t)P.nbox * (128 + 32 * (size_t)P.nc) +
                     (size_t)P.nleaf * 2048 + (1 << 20);
    P.scratch.hint = (size_t)n * 40 + (size_t)P.nbox * 64 + (1 << 20);

    // box point ranges depend on n and the level only
    std::vector<int32_t> hb(P.nbox), hc(P.nbox);
    hb[0] = 0;
    hc[0] = (int32_t)n;
    for (int64_t g = 0; g < P.nbox - P.nleaf; g++) {
        const int32_t k = hc[g] / 2;
        hb[2 * g + 1] = hb[g];
        hc[2 * g + 1] = k;
        hb[2 * g + 2] = hb[g] + k;
        hc[2 * g + 2] = hc[g] - k;
    }
    const size_t nb = (size_t)P.nbox;
    P.x = (double *)fmm::palloc(P, n * 8);
    P.y = (double *)fmm::palloc(P, n * 8);
    P.z = (double *)fmm::palloc(P, n * 8);
    P.perm = (int32_t *)fmm::palloc(P, n * 4);
    P.begin = (int32_t *)fmm::palloc(P, nb * 4);
    P.count = (int32_t *)fmm::palloc(P, nb * 4);
    P.lo = (double *)fmm::palloc(P, nb * 24);
    P.hi = (double *)fmm::palloc(P, nb * 24);
    P.centre = (double *)fmm::palloc(P, nb * 24);
    P.radius = (double *)fmm::palloc(P, nb * 8);
    P.plane = (double *)fmm::palloc(P, nb * 8);
    P.axis = (int32_t *)fmm::palloc(P, nb * 4);
    P.d_err = (int *)fmm::palloc(P, 16);
    if (!P.x || !P.y || !P.z || !P.perm || !P.begin || !P.count || !P.lo || !P.hi || !P.centre ||
        !P.radius || !P.plane || !P.axis || !P.d_err)
        return fail(FMM_ENOMEM);
    if (P.profile)
        for (int s = 0; s < FMM_NSTAGES; s++)
            for (int k = 0; k < 2; k++)
                if (cudaEventCreate(&P.ev[s][k]) != cudaSuccess) return fail(cuda_status(cudaGetLastError()));
    cudaMemcpyAsync(P.begin, hb.data(), nb * 4, cudaMemcpyHostToDevice, P.stream);
    cudaMemcpyAsync(P.count, hc.data(), nb * 4, cudaMemcpyHostToDevice, P.stream);
    cudaMemsetAsync(P.plane, 0, nb * 8, P.stream);
    cudaMemsetAsync(P.d_err, 0, 16, P.stream);

    const void *pts = points;
    void *staged = nullptr;
    const size_t pbytes = (size_t)n * 3 * dsize(dtype);
    if (!is_device_ptr(points)) {
        staged = fmm::dalloc(P, pbytes);
        if (!staged) return fail(FMM_ENOMEM);
        cudaMemcpyAsync(staged, points, pbytes, cudaMemcpyHostToDevice, P.stream);
        pts = staged;
    }
    fmm::stage_mark(P, FMM_STAGE_TREE, 0);
    cudaError_t e = fmm::tree_build(P, pts, dtype);
    if (e == cudaSuccess && P.tight) e = fmm::tight_geometry(P);
    fmm::stage_mark(P, FMM_STAGE_TREE, 1);
    if (staged) fmm::dfree(P, staged, pbytes);
    if (e != cudaSuccess) return fail(cuda_status(e));
    int herr = 0;
    cudaMemcpyAsync(&herr, P.d_err, 4, cudaMemcpyDeviceToHost, P.stream);
    e = cudaStreamSynchronize(P.stream);
    if (e != cudaSuccess) return fail(cuda_status(e));
    if (herr & 1) return fail(FMM_ENONFINITE);
    if (herr & 4) return fail(FMM_EINVAL);  // a point lies outside the given root cell
    if (herr) return fail(FMM_EINTERNAL);  // the partition's consistency check failed

    fmm::stage_mark(P, FMM_STAGE_LISTS, 0);
    e = fmm::lists_build(P);
    fmm::stage_mark(P, FMM_STAGE_LISTS, 1);
    if (P.capacity_exceeded) return fail(FMM_ECAPACITY);
    if (e != cudaSuccess) return fail(cuda_status(e));

    e = fmm::m2l_setup(P);
    if (e != cudaSuccess) return fail(cuda_status(e));
    if (P.prec == FMM_PREC_MIXED) {
        e = fmm::mixed_setup(P);
        if (e == cudaSuccess) e = fmm::m2l_f32_setup(P);
        if (e != cudaSuccess) return fail(cuda_status(e));
    }
    P.q = (double *)fmm::palloc(P, n * 8);
    P.far_phi = (double *)fmm::palloc(P, n * 8);
    P.far_E = (double *)fmm::palloc(P, n * 24);
    P.M = (double2 *)fmm::palloc(P, nb * P.nc * sizeof(double2));
    P.L = (double2 *)fmm::palloc(P, nb * P.nc * sizeof(double2));
    if (!P.q || !P.far_phi || !P.far_E || !P.M || !P.L) return fail(FMM_ENOMEM);
    e = cudaStreamSynchronize(P.stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(cuda_status(e));
    fmm::arena_release(P, P.scratch);  // temporaries of the build, stream-ordered
    *out = H;
    return FMM_OK;
}

int fmm_eval(fmm_plan_t plan, const void *charges, void *potentials, void *fields, void *stream) {
    if (!plan || !charges || !potentials) return FMM_EINVAL;
    if (fmm::ptr_kind(charges) < 0 || fmm::ptr_kind(potentials) < 0 || fmm::ptr_kind(fields) < 0)
        return FMM_EINVAL;
    Plan &P = plan->P;
    P.full_upward = P.ext_active = false;  // a whole evaluation: nothing from other ranks
    P.stream = (cudaStream_t)stream;
    const size_t es = dsize(P.dtype), n = (size_t)P.n;
    const bool dq = is_device_ptr(charges), dp = is_device_ptr(potentials),
               df = !fields || is_device_ptr(fields);
    const size_t need = (dq ? 0 : n * es) + (dp ? 0 : n * es) + (df ? 0 : 3 * n * es);
    if (need > P.stage_bytes) {
        void *s = fmm::palloc(P, need);
        if (!s) return FMM_ENOMEM;
        P.stage = s;
        P.stage_bytes = need;
    }
    char *sp = (char *)P.stage;
    const void *q = charges;
    void *pot = potentials, *fld = fields;
    if (!dq) {
        cudaMemcpyAsync(sp, charges, n * es, cudaMemcpyHostToDevice, P.stream);
        q = sp;
        sp += n * es;
    }
    if (!dp) {
        pot = sp;
        sp += n * es;
    }
    if (!df) fld = sp;
    cudaError_t e = fmm::eval_expansions(P, q, P.dtype);
    if (e == cudaSuccess) e = fmm::eval_p2p(P, pot, fld, P.dtype);
    if (e != cudaSuccess) return cuda_status(e);
    if (!dp) cudaMemcpyAsync(potentials, pot, n * es, cudaMemcpyDeviceToHost, P.stream);
    if (!df) cudaMemcpyAsync(fields, fld, 3 * n * es, cudaMemcpyDeviceToHost, P.stream);
    if (!dp || !df || !dq) {
        e = cudaStreamSynchronize(P.stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return cuda_status(cudaGetLastError());
}

int fmm_eval_check(fmm_plan_t plan) {
    if (!plan) return FMM_EINVAL;
    Plan &P = plan->P;
    int herr[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(herr, P.d_err, 8, cudaMemcpyDeviceToHost, P.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P.stream);
    if (e != cudaSuccess) return cuda_status(e);
    return herr[1] & 16 ? FMM_ETIMEDOUT : FMM_OK;
}

void fmm_destroy(fmm_plan_t plan) {
    if (!plan) return;
    release(plan->P);
    delete plan;
}

int fmm_direct(const void *points, const void *charges, int64_t n, int dtype,
               const int64_t *targets, int64_t ntargets, void *potentials, void *fields,
               void *stream) {
    if (!points || !charges || !targets || !potentials || n < 1 || ntargets < 0) return FMM_EINVAL;
    if (dtype != FMM_F64 && dtype != FMM_F32) return FMM_EINVAL;
    if (fmm::ptr_kind(points) < 0 || fmm::ptr_kind(charges) < 0 || fmm::ptr_kind(targets) < 0 ||
        fmm::ptr_kind(potentials) < 0 || fmm::ptr_kind(fields) < 0)
        return FMM_EINVAL;
    if (ntargets == 0) return FMM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = dsize(dtype);
    const void *a[3] = {points, charges, targets};
    const size_t bytes[3] = {(size_t)n * 3 * es, (size_t)n * es, (size_t)ntargets * 8};
    const size_t obytes[2] = {(size_t)ntargets * es, (size_t)ntargets * 3 * es};
    void *dev[3] = {nullptr, nullptr, nullptr}, *odev[2] = {nullptr, nullptr};
    const void *use[3];
    void *ouse[2] = {potentials, fields};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 3 && e == cudaSuccess; i++) {
        use[i] = a[i];
        if (!is_device_ptr(a[i])) {
            e = cudaMallocAsync(&dev[i], bytes[i], st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dev[i], a[i], bytes[i], cudaMemcpyHostToDevice, st);
            use[i] = dev[i];
        }
    }
    for (int i = 0; i < 2 && e == cudaSuccess; i++) {
        if (ouse[i] && !is_device_ptr(ouse[i])) {
            e = cudaMallocAsync(&odev[i], obytes[i], st);
            ouse[i] = odev[i];
        }
    }
    if (e == cudaSuccess)
        e = fmm::direct_run(use[0], use[1], n, dtype, (const int64_t *)use[2], ntargets, ouse[0],
                            ouse[1], st);
    if (e == cudaSuccess && odev[0]) e = cudaMemcpyAsync(potentials, odev[0], obytes[0], cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && odev[1]) e = cudaMemcpyAsync(fields, odev[1], obytes[1], cudaMemcpyDeviceToHost, st);
    for (int i = 0; i < 3; i++)
        if (dev[i]) cudaFreeAsync(dev[i], st);
    for (int i = 0; i < 2; i++)
        if (odev[i]) cudaFreeAsync(odev[i], st);
    if (odev[0] || odev[1]) {
        cudaError_t e2 = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    return cuda_status(e);
}

void fmm_batch_destroy(fmm_batch_t b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaEvent_t e : b->events) cudaEventDestroy(e);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    if (b->own) cudaStreamDestroy(b->own);
    fmm::batch_release(b->run);
    cudaGetLastError();
    delete b;
}

int fmm_batch_create(const fmm_plan_t *plans, int nplans, const void *const *charges,
                     void *const *potentials, void *const *fields, int nstreams, void *stream,
                     fmm_batch_t *out) {
    if (out) *out = nullptr;
    if (!out || !plans || !charges || !potentials || nplans < 1 || nstreams < 0 || nstreams > 64)
        return FMM_EINVAL;
    for (int i = 0; i < nplans; i++) {
        if (!plans[i] || !is_device_ptr(charges[i]) || !is_device_ptr(potentials[i])) return FMM_EINVAL;
        if (fields && fields[i] && !is_device_ptr(fields[i])) return FMM_EINVAL;
    }
    fmm_batch_s *b = new (std::nothrow) fmm_batch_s();
    if (!b) return FMM_ENOMEM;
    cudaError_t e = cudaSuccess;
    cudaStream_t s0 = (cudaStream_t)stream;
    if (!s0) e = cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking), s0 = b->own;
    std::vector<const Plan *> pl(nplans);
    for (int i = 0; i < nplans; i++) pl[i] = &plans[i]->P;
    bool fused = false;
    if (e == cudaSuccess && fmm::batch_eligible(pl.data(), nplans)) {
        // every system in one launch per stage; a batch whose block counts
        // overflow the int32 offset tables takes the per-plan graph instead
        e = fmm::batch_setup(pl.data(), nplans, charges, potentials, fields, b->run, s0);
        if (e == cudaErrorInvalidValue) {
            cudaGetLastError();
            e = cudaSuccess;
        } else {
            fused = true;
            if (e == cudaSuccess) e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                e = fmm::batch_enqueue(b->run, s0);
                cudaError_t e2 = cudaStreamEndCapture(s0, &b->graph);
                if (e == cudaSuccess) e = e2;
            }
            b->fused = true;
        }
    }
    if (e == cudaSuccess && !fused) {
        // per-plan evaluations on forked branches of the graph
        const int K = std::min(nstreams ? nstreams : 16, nplans);
        for (int k = 0; k < K && e == cudaSuccess; k++) {
            cudaStream_t s;
            e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            if (e == cudaSuccess) b->streams.push_back(s);
        }
        for (int k = 0; k <= K && e == cudaSuccess; k++) {
            cudaEvent_t ev;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) b->events.push_back(ev);
        }
        if (e == cudaSuccess) e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaEventRecord(b->events[K], s0);  // fork
            for (int k = 0; k < K; k++) cudaStreamWaitEvent(b->streams[k], b->events[K], 0);
            for (int i = 0; i < nplans && e == cudaSuccess; i++) {
                Plan &P = plans[i]->P;
                const cudaStream_t keep = P.stream;
                const bool prof = P.profile;
                P.stream = b->streams[i % K];
                P.profile = false;
                P.full_upward = P.ext_active = false;
                e = fmm::eval_expansions(P, charges[i], P.dtype);
                if (e == cudaSuccess) e = fmm::eval_p2p(P, potentials[i], fields ? fields[i] : nullptr, P.dtype);
                P.stream = keep;
                P.profile = prof;
            }
            for (int k = 0; k < K; k++) {  // join
                cudaEventRecord(b->events[k], b->streams[k]);
                cudaStreamWaitEvent(s0, b->events[k], 0);
            }
            cudaError_t e2 = cudaStreamEndCapture(s0, &b->graph);
            if (e == cudaSuccess) e = e2;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e == cudaSuccess) {
        size_t nn = 0;
        e = cudaGraphGetNodes(b->graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (e == cudaSuccess && nn) e = cudaGraphGetNodes(b->graph, nodes.data(), &nn);
        for (size_t i = 0; i < nn && e == cudaSuccess; i++) {
            cudaGraphNodeType t;
            e = cudaGraphNodeGetType(nodes[i], &t);
            if (e == cudaSuccess && t == cudaGraphNodeTypeKernel) b->kernels++;
        }
    }
    if (e != cudaSuccess) {
        fmm_batch_destroy(b);
        return cuda_status(e);
    }
    *out = b;
    return FMM_OK;
}

int fmm_batch_info(fmm_batch_t b, int64_t *kernels, int *fused) {
    if (!b) return FMM_EINVAL;
    if (kernels) *kernels = b->kernels;
    if (fused) *fused = b->fused ? 1 : 0;
    return FMM_OK;
}

int fmm_batch_launch(fmm_batch_t b, void *stream) {
    if (!b || !b->exec) return FMM_EINVAL;
    return cuda_status(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
}

int fmm_plan_stats(fmm_plan_t plan, fmm_stats *out) {
    if (!plan || !out) return FMM_EINVAL;
    const Plan &P = plan->P;
    std::memset(out, 0, sizeof(*out));
    out->n = P.n;
    out->nbox = P.nbox;
    out->nleaf = P.nleaf;
    out->levels = P.B;
    out->p = P.p;
    out->prec = P.prec;
    out->dtype = P.dtype;
    out->theta = P.theta;
    for (int l = 0; l <= P.B; l++) {
        out->weak_pairs_level[l] = P.nweak[l];
        out->weak_pairs += P.nweak[l];
    }
    out->strong_leaf_pairs = P.nstrong[P.B];
    out->p2p_units = P.p2p_nunits;
    out->p2p_partial_slots = P.p2p_nparts;
    unsigned long long work = 0;
    if (P.p2p_work_dev) {
        cudaError_t e = cudaStreamSynchronize(P.stream);
        if (e == cudaSuccess) e = cudaMemcpy(&work, P.p2p_work_dev, 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_status(e);
    }
    out->p2p_interactions = (int64_t)work;
    return FMM_OK;
}

int fmm_plan_tree(fmm_plan_t plan, int64_t *perm, int64_t *begin, int64_t *count, double *lo,
                  double *hi, double *centre, double *radius, int32_t *axis, double *plane) {
    if (!plan) return FMM_EINVAL;
    Plan &P = plan->P;
    cudaError_t e = cudaStreamSynchronize(P.stream);
    const size_t nb = (size_t)P.nbox, n = (size_t)P.n;
    if (e == cudaSuccess && perm) {
        std::vector<int32_t> t(n);
        e = cudaMemcpy(t.data(), P.perm, n * 4, cudaMemcpyDeviceToHost);
        for (size_t i = 0; i < n; i++) perm[i] = t[i];
    }
    if (e == cudaSuccess && (begin || count)) {
        std::vector<int32_t> b(nb), c(nb);
        e = cudaMemcpy(b.data(), P.begin, nb * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(c.data(), P.count, nb * 4, cudaMemcpyDeviceToHost);
        for (size_t i = 0; i < nb; i++) {
            if (begin) begin[i] = b[i];
            if (count) count[i] = c[i];
        }
    }
    if (e == cudaSuccess && lo) e = cudaMemcpy(lo, P.lo, nb * 24, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && hi) e = cudaMemcpy(hi, P.hi, nb * 24, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && centre) e = cudaMemcpy(centre, P.centre, nb * 24, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && radius) e = cudaMemcpy(radius, P.radius, nb * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && axis) e = cudaMemcpy(axis, P.axis, nb * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && plane) e = cudaMemcpy(plane, P.plane, nb * 8, cudaMemcpyDeviceToHost);
    return cuda_status(e);
}

int fmm_plan_list(fmm_plan_t plan, int level, int kind, int64_t *ptr, int32_t *src) {
    if (!plan || !ptr || (kind != 0 && kind != 1)) return FMM_EINVAL;
    Plan &P = plan->P;
    if (level < 0 || level > P.B) return FMM_EINVAL;
    cudaError_t e = cudaStreamSynchronize(P.stream);
    const int64_t nt = (int64_t)1 << level;
    std::vector<int32_t> t(nt + 1);
    const int32_t *dp = kind == 0 ? P.wptr[level] : P.sptr[level];
    const int32_t *ds = kind == 0 ? P.wsrc[level] : P.ssrc[level];
    if (e == cudaSuccess) e = cudaMemcpy(t.data(), dp, (nt + 1) * 4, cudaMemcpyDeviceToHost);
    for (int64_t i = 0; i <= nt; i++) ptr[i] = t[i];
    if (e == cudaSuccess && src && t[nt] > 0)
        e = cudaMemcpy(src, ds, (size_t)t[nt] * 4, cudaMemcpyDeviceToHost);
    return cuda_status(e);
}

int fmm_eval_expansions(fmm_plan_t plan, int which, double *out) {
    if (!plan || !out || (which != 0 && which != 1)) return FMM_EINVAL;
    Plan &P = plan->P;
    cudaError_t e = cudaStreamSynchronize(P.stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(out, which == 0 ? P.M : P.L, (size_t)P.nbox * P.nc * sizeof(double2),
                       cudaMemcpyDeviceToHost);
    return cuda_status(e);
}

}  // extern "C"
