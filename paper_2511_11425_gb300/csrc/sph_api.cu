// sph_api.cu -- the C ABI declared in include/sph.h: context management and
// host orchestration of the kernels.  Every entry point queues its kernels on
// the caller's stream, then reads the device status word back (one small
// device-to-host copy + stream synchronisation) and turns it into a
// sph_status.  No exception, abort or device trap crosses the ABI.
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>

#include "sph_internal.cuh"

using namespace sph;

struct sph_ctx {
    Ctx c;
    double *hbuf = nullptr;  // pinned host scratch (dts, conserved totals)
};

namespace {

sph_status failf(Ctx &c, sph_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c.err = buf;
    return s;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return failf(c, SPH_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t count)
{
    return cudaMalloc((void **)p, sizeof(T) * (count > 0 ? count : 1));
}

void free_ctx(Ctx &c)
{
    void *ptrs[] = {c.st, c.dts, c.dtmin, c.morton_box, c.bbox_part, c.cons_part, c.cons_out,
                    c.keys[0], c.keys[1], c.vals[0], c.vals[1], c.hist, c.digit_tot, c.tmp, c.origin,
                    c.node, c.pm, c.fpos, c.fvel, c.fth, c.acc, c.acc2, c.rho_old, c.h_seed,
                    c.list_start, c.list_cnt, c.list, c.redo, c.gflag, c.mirror};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c.st_host) cudaFreeHost(c.st_host);
    if (c.ev0) cudaEventDestroy(c.ev0);
    if (c.ev1) cudaEventDestroy(c.ev1);
    for (cudaEvent_t e : c.kev)
        if (e) cudaEventDestroy(e);
}

int ilog2_ceil(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

bool particles_ok(const sph_particles *p)
{
    if (!p) return false;
    if (p->n == 0) return true;  // empty arrays may be NULL
    const void *ptrs[] = {p->x[0], p->x[1], p->x[2], p->v[0], p->v[1], p->v[2], p->u, p->m,
                          p->h, p->rho, p->omega, p->a[0], p->a[1], p->a[2], p->dudt_h,
                          p->dudt_av, p->divv, p->dt_i, p->nngb, p->iters, p->id};
    for (const void *q : ptrs)
        if (!q) return false;
    return p->n >= 0;
}

sph_status begin(sph_ctx *ctx, cudaStream_t s)
{
    Ctx &c = ctx->c;
    c.err.clear();
    CK(cudaMemsetAsync(c.st, 0, sizeof(DevStatus), s));
    CK(cudaEventRecord(c.ev0, s));
    return SPH_OK;
}

// read the device status back; translate the first kernel error
sph_status finish(sph_ctx *ctx, cudaStream_t s, float *ms)
{
    Ctx &c = ctx->c;
    CK(cudaGetLastError());
    CK(cudaEventRecord(c.ev1, s));
    CK(cudaMemcpyAsync(c.st_host, c.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ctx->hbuf, c.dts, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (ms) cudaEventElapsedTime(ms, c.ev0, c.ev1);
    const DevStatus &h = *c.st_host;
    switch (h.code) {
    case ST_OK: return SPH_OK;
    case ST_ARG:
        return failf(c, SPH_ERR_ARG, "particle %d: smoothing length reached half a periodic box "
                     "length (minimum image no longer unique)", h.detail);
    case ST_CAPACITY:
        return failf(c, SPH_ERR_CAPACITY, "bucket %d: more than %d bounds-tree nodes or source "
                     "buckets overlap its bounds", h.detail, kWalkCap);
    case ST_NOCONV:
        return failf(c, SPH_ERR_NOCONV, "particle %d: Newton iteration on h did not converge in "
                     "%d iterations", h.detail, c.prm.max_newton);
    case ST_NONFINITE:
        return failf(c, SPH_ERR_NONFINITE, "non-finite value at index %d", h.detail);
    case ST_TIMEOUT: return failf(c, SPH_ERR_TIMEOUT, "device wait timed out (%d)", h.detail);
    default: return failf(c, SPH_ERR_CUDA, "unknown device status %d", h.code);
    }
}

cudaError_t grow_list(Ctx &c, int64_t need)
{
    int64_t cap = need + need / 2 + 1024;
    if (c.list) cudaFree(c.list);
    c.list = nullptr;
    c.list_cap = 0;
    cudaError_t e = cudaMalloc((void **)&c.list, sizeof(unsigned) * (size_t)cap);
    if (e == cudaSuccess) c.list_cap = cap;
    return e;
}

void set_geometry(Ctx &c, int64_t n)
{
    KParams &k = c.kp;
    k.n = (int)n;
    k.nb = (int)((n + kBucket - 1) / kBucket);
    k.logP = ilog2_ceil(k.nb > 0 ? k.nb : 1);
    k.P = 1 << k.logP;
    k.logG = k.logP < 3 ? k.logP : 3;  // groups of 8 buckets (256 particles)
    k.G = 1 << k.logG;
    k.ng = (k.nb + k.G - 1) / k.G;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" sph_status sph_create(const sph_params *prm, int64_t capacity, sph_ctx **out)
{
    if (!prm || !out || capacity < 0 || capacity > (int64_t)0x7fffffff - 64) return SPH_ERR_ARG;
    *out = nullptr;
    if (prm->kernel < 0 || prm->kernel > 3 || !(prm->gamma > 1.0) || !(prm->n_ngb > 0.0) ||
        prm->max_newton < 1 || prm->max_newton > 255 || !(prm->h_rel_tol > 0.0) ||
        !(prm->list_margin >= 0.0) || !(prm->eta_courant > 0.0) || !(prm->eta_acc > 0.0) ||
        !(prm->alpha >= 0.0) || !(prm->beta >= 0.0) || !(prm->eps_av > 0.0) ||
        (prm->energy_mode != SPH_ENERGY_PDV && prm->energy_mode != SPH_ENERGY_ISENTROPIC))
        return SPH_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(prm->box_hi[a] > prm->box_lo[a]) || !std::isfinite(prm->box_lo[a]) ||
            !std::isfinite(prm->box_hi[a]))
            return SPH_ERR_ARG;
    sph_ctx *ctx = new (std::nothrow) sph_ctx;
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    c.prm = *prm;
    c.capacity = capacity;
    cudaGetDevice(&c.device);
    KParams &k = c.kp;
    std::memset(&k, 0, sizeof k);
    k.kernel = prm->kernel;
    k.energy_mode = prm->energy_mode;
    k.max_newton = prm->max_newton;
    double maxext = 0.0, maxabs = 0.0, hcap = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double L = prm->box_hi[a] - prm->box_lo[a];
        k.periodic[a] = prm->periodic[a] ? 1 : 0;
        k.L[a] = (float)L;
        k.invL[a] = (float)(1.0 / L);
        k.halfL[a] = (float)(0.5 * L);
        k.lo[a] = prm->box_lo[a];
        k.hi[a] = prm->box_hi[a];
        maxext = fmax(maxext, L);
        maxabs = fmax(maxabs, fmax(fabs(prm->box_lo[a]), fabs(prm->box_hi[a])));
        if (k.periodic[a]) hcap = fmin(hcap, 0.5 * L);
    }
    k.n_ngb = (float)prm->n_ngb;
    k.gamma = (float)prm->gamma;
    k.alpha = (float)prm->alpha;
    k.beta = (float)prm->beta;
    k.eps_av = (float)prm->eps_av;
    k.eta_courant = (float)prm->eta_courant;
    k.eta_acc = (float)prm->eta_acc;
    k.h_rel_tol = (float)prm->h_rel_tol;
    k.margin = (float)prm->list_margin;
    k.hcap = (float)hcap;
    k.q = std::ldexp(1.0, (int)std::floor(std::log2(maxext)) - 20);
    k.inv_q = 1.0 / k.q;
    k.qf = (float)k.q;
    for (int a = 0; a < 3; ++a) {
        k.Ld[a] = prm->box_hi[a] - prm->box_lo[a];
        k.invLd[a] = 1.0 / k.Ld[a];
    }
    k.eps_abs = (float)(4.0 * std::ldexp(1.0, -23) * fmax(maxext, maxabs));

    int64_t cap = capacity > 0 ? capacity : 1;
    c.nb_cap = (int)((cap + kBucket - 1) / kBucket);
    c.P_cap = 1 << ilog2_ceil(c.nb_cap);
    int ntiles = (int)((cap + kSortTile - 1) / kSortTile);
    sph_status rc = SPH_OK;
#define AL(ptr, cnt)                                                                         \
    do {                                                                                     \
        if (rc == SPH_OK && dalloc(&(ptr), (size_t)(cnt)) != cudaSuccess) {                   \
            rc = failf(c, SPH_ERR_CUDA, "cudaMalloc of %s failed", #ptr);                    \
        }                                                                                    \
    } while (0)
    AL(c.st, 1);
    AL(c.dts, 2);
    AL(c.dtmin, 1);
    AL(c.morton_box, 6);
    AL(c.bbox_part, 152 * 6);
    AL(c.cons_part, 304 * 9);
    AL(c.cons_out, 16);
    AL(c.keys[0], cap);
    AL(c.keys[1], cap);
    AL(c.vals[0], cap);
    AL(c.vals[1], cap);
    AL(c.hist, (size_t)256 * ntiles);
    AL(c.digit_tot, 256);
    {
        char *t = nullptr;
        AL(t, (size_t)112 * cap);
        c.tmp = t;
    }
    AL(c.origin, (size_t)3 * c.nb_cap);
    AL(c.node, (size_t)8 * c.P_cap);
    AL(c.pm, cap);
    AL(c.fpos, cap);
    AL(c.fvel, cap);
    AL(c.fth, cap);
    AL(c.acc, cap);
    AL(c.acc2, cap);
    AL(c.rho_old, cap);
    AL(c.h_seed, cap);
    AL(c.list_start, c.nb_cap);
    AL(c.gflag, c.nb_cap);
    AL(c.list_cnt, c.nb_cap);
    AL(c.redo, (size_t)2 * c.nb_cap);
#undef AL
    if (rc == SPH_OK && grow_list(c, (int64_t)c.nb_cap * 96) != cudaSuccess)
        rc = failf(c, SPH_ERR_CUDA, "cudaMalloc of the interaction lists failed");
    if (rc == SPH_OK && cudaMallocHost((void **)&c.st_host, sizeof(DevStatus)) != cudaSuccess)
        rc = SPH_ERR_CUDA;
    if (rc == SPH_OK && cudaMallocHost((void **)&ctx->hbuf, 32 * sizeof(double)) != cudaSuccess)
        rc = SPH_ERR_CUDA;
    if (rc == SPH_OK && (cudaEventCreate(&c.ev0) != cudaSuccess ||
                         cudaEventCreate(&c.ev1) != cudaSuccess ||
                         cudaEventCreate(&c.kev[0]) != cudaSuccess ||
                         cudaEventCreate(&c.kev[1]) != cudaSuccess ||
                         cudaEventCreate(&c.kev[2]) != cudaSuccess))
        rc = SPH_ERR_CUDA;
    if (rc == SPH_OK && cudaMemset(c.dts, 0, 2 * sizeof(double)) != cudaSuccess) rc = SPH_ERR_CUDA;
    if (rc == SPH_OK && cudaDeviceSynchronize() != cudaSuccess) rc = SPH_ERR_CUDA;
    if (rc != SPH_OK) {
        free_ctx(c);
        if (ctx->hbuf) cudaFreeHost(ctx->hbuf);
        delete ctx;
        return rc;
    }
    *out = ctx;
    return SPH_OK;
}

extern "C" void sph_destroy(sph_ctx *ctx)
{
    if (!ctx) return;
    cudaDeviceSynchronize();
    free_ctx(ctx->c);
    if (ctx->hbuf) cudaFreeHost(ctx->hbuf);
    delete ctx;
}

extern "C" sph_status sph_build_cells(sph_ctx *ctx, sph_particles *p, void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (!particles_ok(p) || p->n > c.capacity)
        return failf(c, SPH_ERR_ARG, "sph_build_cells: NULL array or n = %lld > capacity %lld",
                     p ? (long long)p->n : -1LL, (long long)c.capacity);
    cudaStream_t s = (cudaStream_t)stream;
    c.cells_valid = c.density_valid = c.forces_valid = false;
    set_geometry(c, p->n);
    c.n_built = p->n;
    if (p->n == 0) {
        c.cells_valid = true;
        return SPH_OK;
    }
    sph_status rc = begin(ctx, s);
    if (rc) return rc;
    CK(launch_build(c, *p, s));
    rc = finish(ctx, s, &c.stats.ms_build);
    if (rc == SPH_OK) c.cells_valid = true;
    return rc;
}

namespace {

// walk + Newton, re-walking buckets whose h left the list coverage
sph_status density_passes(sph_ctx *ctx, sph_particles *p, cudaStream_t s)
{
    Ctx &c = ctx->c;
    unsigned long long dpairs = 0, dcand = 0;
    int maxit = 0, relists = 0;
    int64_t entries = 0;
    float ms_walk = 0.f, ms_kernel = 0.f;
    const unsigned *ids = nullptr;  // group ids of a re-walk pass (NULL: all groups)
    int nids = c.kp.ng;
    for (int round = 0; round < 12; ++round) {
        sph_status rc = SPH_OK;
        for (int attempt = 0; attempt < 3; ++attempt) {
            rc = begin(ctx, s);
            if (rc) return rc;
            CK(cudaEventRecord(c.kev[0], s));
            CK(launch_walk(c, *p, WALK_DENSITY, ids, nids, c.h_seed, s));
            CK(cudaEventRecord(c.kev[1], s));
            CK(launch_density(c, *p, c.h_seed, ids, nids, 0, 0, nullptr, nullptr, s));
            CK(cudaEventRecord(c.kev[2], s));
            rc = finish(ctx, s, nullptr);
            float t01 = 0.f, t12 = 0.f;
            cudaEventElapsedTime(&t01, c.kev[0], c.kev[1]);
            cudaEventElapsedTime(&t12, c.kev[1], c.kev[2]);
            ms_walk += t01;
            ms_kernel += t12;
            if ((int64_t)c.st_host->list_need <= c.list_cap) break;
            CK(grow_list(c, (int64_t)c.st_host->list_need));
            c.err.clear();
        }
        if (rc) return rc;
        dpairs += c.st_host->density_pairs;
        dcand += c.st_host->density_cand;
        maxit = maxit > c.st_host->max_iters ? maxit : c.st_host->max_iters;
        entries += c.st_host->list_need;
        unsigned nredo = c.st_host->redo_count;
        if (nredo == 0) {
            c.stats.density_pairs = dpairs;
            c.stats.density_candidates = dcand;
            c.stats.max_newton_iters = maxit;
            c.stats.relists = relists;
            c.stats.list_entries_density = entries;
            c.stats.ms_walk = ms_walk;
            c.stats.ms_density_kernel = ms_kernel;
            return SPH_OK;
        }
        relists += (int)nredo;
        // redo ids were written into the half of c.redo not being read
        ids = (ids == c.redo) ? c.redo + c.nb_cap : c.redo;
        nids = (int)nredo;
    }
    return failf(c, SPH_ERR_NOCONV, "smoothing lengths kept leaving the interaction-list "
                 "coverage after 12 re-walks");
}

}  // namespace

extern "C" sph_status sph_density_h(sph_ctx *ctx, sph_particles *p, const float *h_seed, void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (!particles_ok(p)) return failf(c, SPH_ERR_ARG, "sph_density_h: NULL array");
    if (!c.cells_valid || p->n != c.n_built)
        return failf(c, SPH_ERR_STATE, "sph_density_h needs sph_build_cells on these particles first");
    if (p->n == 0) {
        c.density_valid = true;
        return SPH_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = sizeof(float) * (size_t)p->n;
    if (c.prm.energy_mode == SPH_ENERGY_ISENTROPIC && c.rho_valid)
        CK(cudaMemcpyAsync(c.rho_old, p->rho, bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c.h_seed, h_seed ? h_seed : p->h, bytes, cudaMemcpyDeviceToDevice, s));
    cudaEvent_t t0 = nullptr;
    cudaEventCreate(&t0);
    cudaEventRecord(t0, s);
    sph_status rc = density_passes(ctx, p, s);
    if (rc) {
        cudaEventDestroy(t0);
        return rc;
    }
    rc = begin(ctx, s);
    if (rc) {
        cudaEventDestroy(t0);
        return rc;
    }
    if (c.prm.energy_mode == SPH_ENERGY_ISENTROPIC && c.rho_valid) CK(launch_isentropic(c, *p, s));
    CK(launch_bob_refit(c, *p, s));
    rc = finish(ctx, s, nullptr);
    cudaEventElapsedTime(&c.stats.ms_density, t0, c.ev1);
    cudaEventDestroy(t0);
    if (rc == SPH_OK) {
        c.density_valid = true;
        c.rho_valid = true;
        c.forces_valid = false;
    }
    return rc;
}

extern "C" sph_status sph_density_at(sph_ctx *ctx, sph_particles *p, const float *h, int64_t cap,
                                     uint32_t *count, int64_t *ids, void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (!particles_ok(p) || !h || cap < 0 || (ids && cap == 0))
        return failf(c, SPH_ERR_ARG, "sph_density_at: bad arguments");
    if (!c.cells_valid || p->n != c.n_built)
        return failf(c, SPH_ERR_STATE, "sph_density_at needs sph_build_cells on these particles first");
    if (p->n == 0) return SPH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(c.h_seed, h, sizeof(float) * (size_t)p->n, cudaMemcpyDeviceToDevice, s));
    sph_status rc = SPH_OK;
    for (int attempt = 0; attempt < 3; ++attempt) {
        rc = begin(ctx, s);
        if (rc) return rc;
        CK(launch_walk(c, *p, WALK_DENSITY, nullptr, c.kp.ng, c.h_seed, s));
        CK(launch_density(c, *p, c.h_seed, nullptr, c.kp.ng, 1, cap, count, ids, s));
        rc = finish(ctx, s, nullptr);
        if ((int64_t)c.st_host->list_need <= c.list_cap) break;
        CK(grow_list(c, (int64_t)c.st_host->list_need));
    }
    c.density_valid = false;
    c.forces_valid = false;
    return rc;
}

extern "C" sph_status sph_forces(sph_ctx *ctx, sph_particles *p, void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (!particles_ok(p)) return failf(c, SPH_ERR_ARG, "sph_forces: NULL array");
    if (!c.density_valid || p->n != c.n_built)
        return failf(c, SPH_ERR_STATE, "sph_forces needs sph_density_h on these particles first");
    if (p->n == 0) {
        c.forces_valid = true;
        return SPH_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    sph_status rc = SPH_OK;
    for (int attempt = 0; attempt < 3; ++attempt) {
        rc = begin(ctx, s);
        if (rc) return rc;
        CK(launch_predict(c, *p, s));
        CK(cudaEventRecord(c.kev[0], s));
        CK(launch_walk(c, *p, WALK_FORCE, nullptr, c.kp.ng, nullptr, s));
        CK(cudaEventRecord(c.kev[1], s));
        CK(launch_forces(c, *p, s));
        CK(cudaEventRecord(c.kev[2], s));
        CK(launch_finalize(c, *p, s));
        rc = finish(ctx, s, &c.stats.ms_forces);
        if ((int64_t)c.st_host->list_need <= c.list_cap) break;
        CK(grow_list(c, (int64_t)c.st_host->list_need));
        c.err.clear();
    }
    if (rc == SPH_OK) {
        c.forces_valid = true;
        c.stats.force_pairs = c.st_host->force_pairs;
        c.stats.force_candidates = c.st_host->force_cand;
        c.stats.list_entries_force = c.st_host->list_need;
        c.stats.force_av_pairs = c.st_host->force_av_pairs;
        float t01 = 0.f, t12 = 0.f;
        cudaEventElapsedTime(&t01, c.kev[0], c.kev[1]);
        cudaEventElapsedTime(&t12, c.kev[1], c.kev[2]);
        c.stats.ms_walk += t01;
        c.stats.ms_force_kernel = t12;
    }
    return rc;
}

extern "C" sph_status sph_kdk_step(sph_ctx *ctx, sph_particles *p, double dt_fixed,
                                   double *dt_used, void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (!particles_ok(p)) return failf(c, SPH_ERR_ARG, "sph_kdk_step: NULL array");
    if (!c.forces_valid || p->n != c.n_built)
        return failf(c, SPH_ERR_STATE, "sph_kdk_step needs sph_forces on these particles first");
    if (!(dt_fixed == dt_fixed) || std::isinf(dt_fixed))
        return failf(c, SPH_ERR_ARG, "sph_kdk_step: dt_fixed must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    if (p->n == 0) {
        if (dt_used) *dt_used = dt_fixed > 0 ? dt_fixed : 0.0;
        return SPH_OK;
    }
    sph_status rc = begin(ctx, s);
    if (rc) return rc;
    CK(launch_kdk(c, *p, dt_fixed, s));
    rc = finish(ctx, s, &c.stats.ms_kdk);
    c.cells_valid = c.density_valid = c.forces_valid = false;
    if (rc == SPH_OK) {
        c.stats.dt_old = ctx->hbuf[0];
        if (dt_used) *dt_used = ctx->hbuf[0];
    }
    return rc;
}

extern "C" sph_status sph_step(sph_ctx *ctx, sph_particles *p, double dt_fixed, double *dt_used,
                               void *stream)
{
    sph_status rc = sph_build_cells(ctx, p, stream);
    if (rc) return rc;
    rc = sph_density_h(ctx, p, nullptr, stream);
    if (rc) return rc;
    rc = sph_forces(ctx, p, stream);
    if (rc) return rc;
    return sph_kdk_step(ctx, p, dt_fixed, dt_used, stream);
}

namespace {
struct ArrDesc {
    size_t off;   // offset of the pointer member in sph_particles
    size_t elem;  // element size
};
const ArrDesc kArrays[] = {
    {offsetof(sph_particles, x) + 0 * sizeof(double *), 8},
    {offsetof(sph_particles, x) + 1 * sizeof(double *), 8},
    {offsetof(sph_particles, x) + 2 * sizeof(double *), 8},
    {offsetof(sph_particles, v) + 0 * sizeof(double *), 8},
    {offsetof(sph_particles, v) + 1 * sizeof(double *), 8},
    {offsetof(sph_particles, v) + 2 * sizeof(double *), 8},
    {offsetof(sph_particles, u), 8},
    {offsetof(sph_particles, m), 4},
    {offsetof(sph_particles, h), 4},
    {offsetof(sph_particles, rho), 4},
    {offsetof(sph_particles, omega), 4},
    {offsetof(sph_particles, a) + 0 * sizeof(float *), 4},
    {offsetof(sph_particles, a) + 1 * sizeof(float *), 4},
    {offsetof(sph_particles, a) + 2 * sizeof(float *), 4},
    {offsetof(sph_particles, dudt_h), 4},
    {offsetof(sph_particles, dudt_av), 4},
    {offsetof(sph_particles, divv), 4},
    {offsetof(sph_particles, dt_i), 4},
    {offsetof(sph_particles, nngb), 2},
    {offsetof(sph_particles, iters), 1},
    {offsetof(sph_particles, id), 8},
};
void *&member(sph_particles &p, const ArrDesc &d)
{
    return *reinterpret_cast<void **>(reinterpret_cast<char *>(&p) + d.off);
}
}  // namespace

extern "C" sph_status sph_step_host(sph_ctx *ctx, sph_host_particles *hp, double dt_fixed,
                                    double *dt_used, int64_t *h2d_bytes, int64_t *d2h_bytes,
                                    void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (!particles_ok(hp) || hp->n > c.capacity)
        return failf(c, SPH_ERR_ARG, "sph_step_host: NULL array or n > capacity");
    cudaStream_t s = (cudaStream_t)stream;
    size_t cap = (size_t)(c.capacity > 0 ? c.capacity : 1);
    if (!c.mirror) {
        size_t total = 0;
        for (const ArrDesc &d : kArrays) total += ((d.elem * cap + 255) / 256) * 256;
        CK(cudaMalloc(&c.mirror, total));
        char *base = (char *)c.mirror;
        for (const ArrDesc &d : kArrays) {
            member(c.dmirror, d) = base;
            base += ((d.elem * cap + 255) / 256) * 256;
        }
    }
    c.dmirror.n = hp->n;
    int64_t moved = 0;
    for (const ArrDesc &d : kArrays) {
        size_t b = d.elem * (size_t)hp->n;
        CK(cudaMemcpyAsync(member(c.dmirror, d), member(*hp, d), b, cudaMemcpyHostToDevice, s));
        moved += (int64_t)b;
    }
    if (h2d_bytes) *h2d_bytes = moved;
    sph_status rc = sph_step(ctx, &c.dmirror, dt_fixed, dt_used, stream);
    if (rc) return rc;
    for (const ArrDesc &d : kArrays) {
        size_t b = d.elem * (size_t)hp->n;
        CK(cudaMemcpyAsync(member(*hp, d), member(c.dmirror, d), b, cudaMemcpyDeviceToHost, s));
    }
    if (d2h_bytes) *d2h_bytes = moved;
    CK(cudaStreamSynchronize(s));
    return SPH_OK;
}

extern "C" sph_status sph_reduce_conserved(sph_ctx *ctx, const sph_particles *p, double out[9],
                                           void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (!particles_ok(p) || !out) return failf(c, SPH_ERR_ARG, "sph_reduce_conserved: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    sph_status rc = begin(ctx, s);
    if (rc) return rc;
    CK(launch_conserved(c, *p, s));
    CK(cudaMemcpyAsync(ctx->hbuf + 8, c.cons_out, 9 * sizeof(double), cudaMemcpyDeviceToHost, s));
    rc = finish(ctx, s, nullptr);
    if (rc == SPH_OK) std::memcpy(out, ctx->hbuf + 8, 9 * sizeof(double));
    return rc;
}

extern "C" sph_status sph_set_dt_old(sph_ctx *ctx, double dt_old)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (!(dt_old >= 0.0) || std::isinf(dt_old)) return failf(c, SPH_ERR_ARG, "dt_old must be >= 0");
    double v[2] = {dt_old, dt_old};
    CK(cudaMemcpy(c.dts, v, sizeof v, cudaMemcpyHostToDevice));
    c.stats.dt_old = dt_old;
    return SPH_OK;
}

extern "C" sph_status sph_get_stats(const sph_ctx *ctx, sph_stats *out)
{
    if (!ctx || !out) return SPH_ERR_ARG;
    *out = ctx->c.stats;
    out->launches = ctx->c.launches;
    return SPH_OK;
}

extern "C" const char *sph_last_error(const sph_ctx *ctx)
{
    return ctx ? ctx->c.err.c_str() : "NULL context";
}

extern "C" const char *sph_version(void) { return "libsph 0.1 (sm_103a)"; }
