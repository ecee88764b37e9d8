// sph_api.cu -- the C ABI declared in include/sph.h: contexts, the layout of
// instances, buckets, groups and trees, and host orchestration of the kernels.
//
// Every phase is queued on the caller's stream without host round trips; an
// entry point ends with ONE device-to-host read of the status word and a
// stream synchronisation, then turns the status into a sph_status.  The same
// queue can be captured once into a CUDA graph and replayed.  No exception,
// abort or device trap crosses the ABI.
#include <algorithm>
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

int ilog2_ceil(int64_t v)
{
    int l = 0;
    while (((int64_t)1 << l) < v) ++l;
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

bool params_ok(const sph_params *prm)
{
    if (!prm) return false;
    if (prm->kernel < 0 || prm->kernel > 3 || !(prm->gamma > 1.0) || !(prm->n_ngb > 0.0) ||
        prm->max_newton < 1 || prm->max_newton > 255 || !(prm->h_rel_tol > 0.0) ||
        !(prm->list_margin >= 0.0) || !(prm->eta_courant > 0.0) || !(prm->eta_acc > 0.0) ||
        !(prm->alpha >= 0.0) || !(prm->beta >= 0.0) || !(prm->eps_av > 0.0) ||
        (prm->energy_mode != SPH_ENERGY_PDV && prm->energy_mode != SPH_ENERGY_ISENTROPIC) ||
        (prm->curve != SPH_CURVE_HILBERT && prm->curve != SPH_CURVE_MORTON) ||
        prm->group_log < 0 || prm->group_log > kGroupLog ||
        !(prm->bucket_cell == 0.0 || prm->bucket_cell >= 1.0) ||
        !(prm->group_cell == 0.0 || prm->group_cell >= 1.0))
        return false;
    if (prm->resort_period < 0 || prm->resort_period > 64) return false;
    if (prm->precision != SPH_PRECISION_MIXED && prm->precision != SPH_PRECISION_FP64) return false;
    if (prm->density_mode != SPH_DENSITY_SUMMED && prm->density_mode != SPH_DENSITY_EVOLVED)
        return false;
    if (prm->density_mode == SPH_DENSITY_EVOLVED && prm->energy_mode != SPH_ENERGY_PDV) return false;
    if (prm->interface_correction != 0 && prm->interface_correction != 1) return false;
    if (prm->interface_correction) {
        // Sec. 2.3.4: not with the evolved density; built for the mixed form
        if (prm->density_mode != SPH_DENSITY_SUMMED || prm->precision != SPH_PRECISION_MIXED)
            return false;
        if (!(prm->ic_alpha >= 0.0) || !std::isfinite(prm->ic_alpha)) return false;
        for (int k = 0; k < 4; ++k)
            if (!(prm->r_gas[k] > 0.0) || !std::isfinite(prm->r_gas[k])) return false;
    }
    const double kb = prm->bucket_cell > 0.0 ? prm->bucket_cell : kKappaBucket;
    const double kg = prm->group_cell > 0.0 ? prm->group_cell : kKappaGroup;
    if (!(kg >= kb) || !std::isfinite(kg)) return false;
    for (int a = 0; a < 3; ++a)
        if (!(prm->box_hi[a] > prm->box_lo[a]) || !std::isfinite(prm->box_lo[a]) ||
            !std::isfinite(prm->box_hi[a]))
            return false;
    return true;
}

// physical parameters of one instance (geometry fields are set by the layout)
Inst inst_params(const sph_params &prm)
{
    Inst I;
    std::memset(&I, 0, sizeof I);
    double maxext = 0.0, maxabs = 0.0, hcap = INFINITY;
    for (int a = 0; a < 3; ++a) {
        const double L = prm.box_hi[a] - prm.box_lo[a];
        I.periodic[a] = prm.periodic[a] ? 1 : 0;
        I.L[a] = (float)L;
        I.invL[a] = (float)(1.0 / L);
        I.lo[a] = prm.box_lo[a];
        I.hi[a] = prm.box_hi[a];
        I.Ld[a] = L;
        I.invLd[a] = 1.0 / L;
        maxext = fmax(maxext, L);
        maxabs = fmax(maxabs, fmax(fabs(prm.box_lo[a]), fabs(prm.box_hi[a])));
        if (I.periodic[a]) hcap = fmin(hcap, 0.5 * L);
    }
    I.gamma = (float)prm.gamma;
    I.alpha = (float)prm.alpha;
    I.beta = (float)prm.beta;
    I.eps_av = (float)prm.eps_av;
    I.eta_courant = (float)prm.eta_courant;
    I.eta_acc = (float)prm.eta_acc;
    I.n_ngb = (float)prm.n_ngb;
    I.curve = prm.curve;
    I.kb = (float)(prm.bucket_cell > 0.0 ? prm.bucket_cell : kKappaBucket);
    I.kg = (float)(prm.group_cell > 0.0 ? prm.group_cell : kKappaGroup);
    I.hcap = (float)hcap;
    I.q = std::ldexp(1.0, (int)std::floor(std::log2(maxext)) - 20);
    I.inv_q = 1.0 / I.q;
    I.qf = (float)I.q;
    // fixed-point positions of the force pairs (units qx = q 2^-kFixShift):
    // bucket-relative coordinates and pair separations stay below 2^31 qx
    // while bucket extents and h stay below fix_lim (checked per launch)
    const double qx = std::ldexp(I.q, -kFixShift);
    I.qx = (float)qx;
    I.inv_qx = (float)(1.0 / qx);
    I.qx2 = (float)(qx * qx);
    I.fix_lim = (float)(0.99 * std::ldexp(qx, 31));
    for (int a = 0; a < 3; ++a)
        I.LQ[a] = I.periodic[a] ? (unsigned)std::llrint((prm.box_hi[a] - prm.box_lo[a]) / qx) : 0u;
    I.eps_abs = (float)(4.0 * std::ldexp(1.0, -23) * fmax(maxext, maxabs));
    // kernel-imbalance normalisation: 1 / (2 pi int_0^1 w(q) q^3 dq), the
    // value at which a particle on a flat interface between two uniform
    // materials has I = 1 (closed forms of the four kernels)
    const double ic_norm[4] = {24.0 / 5.0, 192.0 / 35.0, 128.0 / 21.0, 140.0 / 31.0};
    I.ic_alpha = (float)(prm.ic_alpha > 0.0 ? prm.ic_alpha : ic_norm[prm.kernel & 3]);
    for (int k = 0; k < 4; ++k) I.r_gas[k] = (float)prm.r_gas[k];
    return I;
}

// sizes the layout of `counts` needs
struct Sizes {
    int64_t n = 0, nb = 0, ng = 0, nodes = 0, refit = 0, cons_blocks = 0;
};

// log2 of the buckets per walk group of an instance
int group_log(const sph_params &prm, int logP)
{
    return std::min(logP, prm.group_log > 0 ? prm.group_log : kGroupLog);
}

Sizes layout_sizes(const std::vector<int64_t> &counts, const std::vector<sph_params> &prm)
{
    Sizes z;
    for (size_t k = 0; k < counts.size(); ++k) {
        const int64_t nk = counts[k];
        const int64_t nb = bucket_slots(nk);
        const int logP = ilog2_ceil(std::max<int64_t>(nb, 1));
        const int64_t P = (int64_t)1 << logP;
        const int logG = group_log(prm[k], logP);
        z.n += nk;
        z.nb += nb;
        z.ng += (nb + (1 << logG) - 1) >> logG;
        z.nodes += 2 * P;
        z.refit += P / 2 + 4;  // one block per 256 nodes of a band, plus the upper bands
        z.cons_blocks = std::max<int64_t>(z.cons_blocks, (nk + kConsChunk - 1) / kConsChunk);
    }
    return z;
}

// allocate every buffer for the sizes `cap`
sph_status allocate(Ctx &c, const Sizes &cap, int ninst)
{
    const int64_t np = std::max<int64_t>(cap.n, 1);
    const int64_t nb = std::max<int64_t>(cap.nb, 1), ng = std::max<int64_t>(cap.ng, 1);
    const int64_t ntiles = (np + kSortTile - 1) / kSortTile;
    sph_status rc = SPH_OK;
#define AL(ptr, cnt)                                                                         \
    do {                                                                                     \
        if (rc == SPH_OK && dalloc(&(ptr), (size_t)(cnt)) != cudaSuccess) {                   \
            rc = failf(c, SPH_ERR_CUDA, "cudaMalloc of %s failed", #ptr);                    \
        }                                                                                    \
    } while (0)
    AL(c.st, 1);
    AL(c.inst, ninst);
    AL(c.dts, 2 * ninst);
    AL(c.dtmin, ninst);
    AL(c.morton_box, kKeyBox * ninst);
    AL(c.bbox_part, (size_t)6 * kBboxChunks * ninst);
    AL(c.cons_part, (size_t)9 * std::max<int64_t>(cap.cons_blocks, 1) * ninst);
    AL(c.cons_out, (size_t)9 * ninst);
    AL(c.pinst, np);
    AL(c.keys[0], np);
    AL(c.keys[1], np);
    AL(c.vals[0], np);
    AL(c.vals[1], np);
    AL(c.hist, (size_t)256 * ntiles);
    AL(c.digit_tot, 256);
    {
        char *t = nullptr;
        AL(t, (size_t)112 * np);
        c.tmp = t;
    }
    AL(c.bstart, nb + 1);
    AL(c.binst, nb);
    AL(c.pad_agg, (np + kPadTile - 1) / kPadTile);
    AL(c.pad_used, ninst);
    AL(c.origin, (size_t)3 * nb);
    AL(c.gfirst, ng);
    AL(c.gflag, ng);
    AL(c.list_cnt, ng);
    AL(c.list_off, ng);
    AL(c.arena_used, 1);
    c.arena_cap = std::max<int64_t>((int64_t)1 << 23, 16 * ng);
    c.arena_alloc = c.arena_cap;
    c.list_slots = ng * kWalkCap;
    if (rc == SPH_OK && ng * kWalkCap + c.arena_cap > (int64_t)0xffffffffLL)
        rc = failf(c, SPH_ERR_CAPACITY, "too many walk groups (%lld) for 32-bit list offsets",
                   (long long)ng);
    AL(c.list, (size_t)ng * kWalkCap + (size_t)c.arena_cap);
    AL(c.redo, (size_t)kRelistRounds * ng);
    AL(c.node, (size_t)4 * std::max<int64_t>(cap.nodes, 2));
    AL(c.refit, std::max<int64_t>(cap.refit, 1));
    AL(c.pm, np);
    AL(c.fpos, np);
    AL(c.fvel, np);
    AL(c.fth, np);
    AL(c.ipos, np);
    if (c.kp.evolved) AL(c.rho_sum, np);
    if (c.kp.ic) {
        AL(c.ic_e, np);
        AL(c.ic_pt, np);
    }
    if (c.kp.fp64) {
        AL(c.pmd, np);
        AL(c.fveld, np);
        AL(c.fthd, np);
        AL(c.acc64, np);
    }
    AL(c.acc, np);
    AL(c.accS, np);
    AL(c.mumax, np);
    AL(c.rho_old, np);
    AL(c.h_seed, np);
#undef AL
    if (rc == SPH_OK && (cudaMallocHost((void **)&c.st_host, sizeof(DevStatus)) != cudaSuccess ||
                         cudaMallocHost((void **)&c.dts_host, sizeof(double) * 2 * ninst) != cudaSuccess ||
                         cudaMallocHost((void **)&c.cons_host, sizeof(double) * 9 * ninst) != cudaSuccess))
        rc = failf(c, SPH_ERR_CUDA, "cudaMallocHost failed");
    if (rc == SPH_OK) {
        for (cudaEvent_t *e : {&c.ev0, &c.ev1, &c.kev[0], &c.kev[1], &c.kev[2], &c.kev[3],
                               &c.kev[4], &c.kev[5]})
            if (cudaEventCreate(e) != cudaSuccess) rc = failf(c, SPH_ERR_CUDA, "cudaEventCreate failed");
        for (cudaEvent_t *e : {&c.fork, &c.join, &c.call0, &c.late_in, &c.out_dens, &c.out_force,
                               &c.out_done})
            if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess)
                rc = failf(c, SPH_ERR_CUDA, "cudaEventCreate failed");
        for (cudaStream_t *st : {&c.side, &c.copy})
            if (cudaStreamCreateWithFlags(st, cudaStreamNonBlocking) != cudaSuccess)
                rc = failf(c, SPH_ERR_CUDA, "cudaStreamCreate failed");
    }
    if (rc == SPH_OK && cudaMemset(c.dts, 0, sizeof(double) * 2 * ninst) != cudaSuccess)
        rc = SPH_ERR_CUDA;
    if (rc == SPH_OK && c.st_host) std::memset(c.st_host, 0, sizeof(DevStatus));
    if (rc == SPH_OK && c.dts_host) std::memset(c.dts_host, 0, sizeof(double) * 2 * ninst);
    c.cons_blocks = (int)std::max<int64_t>(cap.cons_blocks, 1);
    return rc;
}

void free_ctx(Ctx &c)
{
    if (c.graph_exec) cudaGraphExecDestroy(c.graph_exec);
    if (c.graph) cudaGraphDestroy(c.graph);
    if (c.graph_exec_r) cudaGraphExecDestroy(c.graph_exec_r);
    if (c.graph_r) cudaGraphDestroy(c.graph_r);
    void *ptrs[] = {c.st, c.inst, c.dts, c.dtmin, c.morton_box, c.bbox_part, c.cons_part,
                    c.pad_agg, c.pad_used,
                    c.cons_out, c.pinst, c.keys[0], c.keys[1], c.vals[0], c.vals[1], c.hist,
                    c.digit_tot, c.tmp, c.bstart, c.binst, c.origin, c.gfirst, c.gflag,
                    c.list_cnt, c.list_off, c.arena_used, c.list, c.redo, c.node, c.refit,
                    c.pm, c.pmd, c.fveld, c.fthd, c.acc64, c.ipos, c.fpos, c.fvel, c.fth,
                    c.acc, c.accS, c.mumax, c.rho_sum, c.ic_e, c.ic_pt, c.rung, c.rmax, c.bact, c.gmark, c.fg_list, c.rho_old, c.h_seed, c.mirror};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    void *mptrs[] = {c.mlp.w, c.mlp.m, c.mlp.v, c.mlp.frag, c.mlp.gpart, c.mlp.loss,
                     c.mlp.seed0, c.mlp.corr, c.mlp.tfeat, c.mlp.th, c.mlp.sx, c.mlp.sy,
                     c.mlp.scount};
    for (void *p : mptrs)
        if (p) cudaFree(p);
    for (void *p : {(void *)c.st_host, (void *)c.dts_host, (void *)c.cons_host})
        if (p) cudaFreeHost(p);
    for (cudaEvent_t e : {c.ev0, c.ev1, c.kev[0], c.kev[1], c.kev[2], c.kev[3], c.kev[4], c.kev[5],
                          c.fork, c.join, c.call0, c.late_in, c.out_dens, c.out_force,
                          c.out_done})
        if (e) cudaEventDestroy(e);
    for (cudaStream_t st : {c.side, c.copy})
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : c.prof.ev)
        if (e) cudaEventDestroy(e);
    c.prof.ev.clear();
    for (int g = 0; g < 2; ++g) {
        for (cudaEvent_t e : c.prof.gev[g])
            if (e) cudaEventDestroy(e);
        c.prof.gev[g].clear();
        c.prof.gphase[g].clear();
    }
}

// lay out instances of the given particle counts (offsets follow the order)
// and upload the index maps; synchronous (only when the layout changes)
sph_status set_layout(Ctx &c, const std::vector<int64_t> &counts)
{
    const int ni = (int)counts.size();
    std::vector<Inst> insts(ni);
    std::vector<int> bstart, binst, gfirst;
    std::vector<unsigned short> pinst;
    std::vector<std::vector<RefitBlock>> bands;
    int64_t off = 0, boff = 0, goff = 0, nbase = 0;
    bool any_open = false;
    for (int k = 0; k < ni; ++k) {
        Inst I = inst_params(c.prm[k]);
        const int64_t nk = counts[k];
        I.off = (int)off;
        I.n = (int)nk;
        I.nb = (int)bucket_slots(nk);
        I.boff = (int)boff;
        I.logP = ilog2_ceil(std::max(I.nb, 1));
        I.P = 1 << I.logP;
        I.logG = group_log(c.prm[k], I.logP);
        I.G = 1 << I.logG;
        I.ng = (I.nb + I.G - 1) >> I.logG;
        I.goff = (int)goff;
        I.nbase = (int)nbase;
        for (int a = 0; a < 3; ++a) any_open = any_open || !I.periodic[a];
        for (int b = 0; b < I.nb; ++b) {  // plain chunks until the first build
            bstart.push_back((int)std::min<int64_t>(I.off + (int64_t)b * kBucket, I.off + nk));
            binst.push_back(k);
        }
        for (int g = 0; g < I.ng; ++g) gfirst.push_back(I.boff + (g << I.logG));
        pinst.insert(pinst.end(), (size_t)nk, (unsigned short)k);
        int lvl = I.logP, band = 0;
        while (lvl > 0) {
            const int levels = std::min(lvl, 8);
            if ((int)bands.size() <= band) bands.emplace_back();
            for (int blk = 0; blk < (1 << (lvl - levels)); ++blk)
                bands[band].push_back(RefitBlock{k, lvl, levels, blk});
            lvl -= levels;
            ++band;
        }
        insts[k] = I;
        off += nk;
        boff += I.nb;
        goff += I.ng;
        nbase += 2 * (int64_t)I.P;
    }
    bstart.push_back((int)off);  // sentinel: one past the last slot
    std::vector<RefitBlock> sched;
    c.refit_band.clear();
    for (auto &b : bands) {
        c.refit_band.push_back((int)b.size());
        sched.insert(sched.end(), b.begin(), b.end());
    }
    int nbits = 30;
    while (((int64_t)1 << (nbits - 30)) < ni) ++nbits;
    KParams &kp = c.kp;
    kp.ninst = ni;
    kp.n = (int)off;
    kp.nb = (int)boff;
    kp.ng = (int)goff;
    kp.nnodes = (int)nbase;
    kp.key_passes = (nbits + 7) / 8;
    kp.any_open = any_open ? 1 : 0;
    c.inst_host = insts;
    int64_t cb = 1;
    for (int64_t nk : counts) cb = std::max<int64_t>(cb, (nk + kConsChunk - 1) / kConsChunk);
    c.cons_blocks = (int)cb;
    CK(cudaMemcpy(c.inst, insts.data(), sizeof(Inst) * ni, cudaMemcpyHostToDevice));
    if (!bstart.empty()) {
        CK(cudaMemcpy(c.bstart, bstart.data(), sizeof(int) * bstart.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c.binst, binst.data(), sizeof(int) * binst.size(), cudaMemcpyHostToDevice));
    }
    if (!gfirst.empty())
        CK(cudaMemcpy(c.gfirst, gfirst.data(), sizeof(int) * gfirst.size(), cudaMemcpyHostToDevice));
    if (!pinst.empty())
        CK(cudaMemcpy(c.pinst, pinst.data(), sizeof(unsigned short) * pinst.size(),
                      cudaMemcpyHostToDevice));
    if (!sched.empty())
        CK(cudaMemcpy(c.refit, sched.data(), sizeof(RefitBlock) * sched.size(),
                      cudaMemcpyHostToDevice));
    c.n_built = off;
    c.order_fresh = false;
    // records of the last kick belong to the old layout
    if (c.mlp.th) CK(cudaMemset(c.mlp.th, 0, sizeof(float) * (size_t)c.capacity));
    return SPH_OK;
}

// add the timed launch groups of the call that just completed to the
// per-phase totals (groups whose events did not complete are dropped)
void prof_collect(Ctx &c)
{
    for (size_t k = 0; k < c.prof.phase.size(); ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c.prof.ev[2 * k], c.prof.ev[2 * k + 1]) == cudaSuccess) {
            c.prof.ms[c.prof.phase[k]] += ms;
            c.prof.launches[c.prof.phase[k]] += 1;
        } else {
            cudaGetLastError();
        }
    }
    c.prof.phase.clear();
}

// the same for the launch groups recorded into captured step `slot`, after
// a replay of it completed
void prof_collect_graph(Ctx &c, int slot)
{
    const std::vector<int> &ph = c.prof.gphase[slot];
    const std::vector<cudaEvent_t> &ev = c.prof.gev[slot];
    for (size_t k = 0; k < ph.size(); ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]) == cudaSuccess) {
            c.prof.ms[ph[k]] += ms;
            c.prof.launches[ph[k]] += 1;
        } else {
            cudaGetLastError();
        }
    }
}

sph_status begin(sph_ctx *ctx, cudaStream_t s)
{
    Ctx &c = ctx->c;
    c.err.clear();
    c.prof.phase.clear();
    CK(cudaMemsetAsync(c.st, 0, sizeof(DevStatus), s));
    return SPH_OK;
}

// queue the status read-back (also recorded into a captured graph)
sph_status queue_status(Ctx &c, cudaStream_t s)
{
    CK(cudaMemcpyAsync(c.st_host, c.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c.dts_host, c.dts, sizeof(double) * 2 * c.kp.ninst, cudaMemcpyDeviceToHost, s));
    return SPH_OK;
}

// wait for the queued work and translate the first kernel error
sph_status settle(sph_ctx *ctx, cudaStream_t s)
{
    Ctx &c = ctx->c;
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    if (!c.prof.phase.empty()) prof_collect(c);
    const DevStatus &h = *c.st_host;
    switch (h.code) {
    case ST_OK: return SPH_OK;
    case ST_ARG:
        return failf(c, SPH_ERR_ARG, "index %d: smoothing length reached half a periodic box "
                     "length, or a bucket left the position grid", h.detail);
    case ST_CAPACITY:
        return failf(c, SPH_ERR_CAPACITY, "group %d: the interaction-list overflow arena "
                     "(%lld entries) is full", h.detail, (long long)c.arena_cap);
    case ST_NOCONV:
        return failf(c, SPH_ERR_NOCONV, "particle %d: Newton iteration on h did not converge in "
                     "%d iterations or %d re-walks", h.detail, c.kp.max_newton, kRelistRounds);
    case ST_NONFINITE:
        return failf(c, SPH_ERR_NONFINITE, "non-finite value at index %d", h.detail);
    default: return failf(c, SPH_ERR_CUDA, "unknown device status %d", h.code);
    }
}

sph_status finish(sph_ctx *ctx, cudaStream_t s)
{
    Ctx &c = ctx->c;
    CK(cudaGetLastError());
    CK(cudaEventRecord(c.ev1, s));
    sph_status rc = queue_status(c, s);
    if (rc) return rc;
    return settle(ctx, s);
}

float elapsed(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        ms = 0.f;
        (void)cudaGetLastError();  // a missing record is not a failure of the step
    }
    return ms;
}

// phase event; under stream capture it must become a record node of the
// graph (a plain record only orders the captured work)
cudaError_t record(const Ctx &c, cudaEvent_t e, cudaStream_t s)
{
    return c.capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                       : cudaEventRecord(e, s);
}

// the step inputs sph_step_host copies in beside the step (v, u, a, du/dt):
// every kernel that reads them comes after this wait.  The event's last
// record is resolved when the wait (or the graph holding it) is launched;
// with no sph_step_host call in flight it has completed and costs nothing.
cudaError_t wait_late_inputs(const Ctx &c, cudaStream_t s)
{
    return cudaStreamWaitEvent(s, c.late_in, c.capturing ? cudaEventWaitExternal : 0);
}

// make sure the layout matches p->n (single-problem contexts follow n)
sph_status ensure_layout(Ctx &c, const sph_particles *p)
{
    if (!particles_ok(p)) return failf(c, SPH_ERR_ARG, "NULL particle array or n < 0");
    if (p->n > c.capacity)
        return failf(c, SPH_ERR_ARG, "n = %lld exceeds the capacity %lld", (long long)p->n,
                     (long long)c.capacity);
    if (c.kp.ic && p->n > 0 && !p->mat)
        return failf(c, SPH_ERR_ARG, "the interface correction needs material ids (p->mat)");
    if (c.prm.size() > 1) {
        if (p->n != c.kp.n)
            return failf(c, SPH_ERR_ARG, "a batch context needs exactly %d particles", c.kp.n);
        return SPH_OK;
    }
    if (p->n != c.n_built || c.inst_host.empty()) return set_layout(c, {p->n});
    return SPH_OK;
}

// ---- phases: queue only ------------------------------------------------------
// fg: a hierarchical substep with FastGas on: after the walk, mark the
// groups of the active particles and of their neighbours, and solve only
// those (the others keep h, rho, Omega of their last pass)
sph_status q_density(Ctx &c, sph_particles *p, const float *h_seed, cudaStream_t s, bool timed,
                     const RungArgs *fg = nullptr)
{
    const size_t bytes = sizeof(float) * (size_t)p->n;
    const bool isen = c.kp.energy_mode == SPH_ENERGY_ISENTROPIC && c.rho_valid;
    if (isen) CK(cudaMemcpyAsync(c.rho_old, p->rho, bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c.h_seed, h_seed ? h_seed : p->h, bytes, cudaMemcpyDeviceToDevice, s));
    // the learned seed's inputs compare h with the seed as given (re-walks
    // overwrite c.h_seed)
    if (c.mlp.seed0 && (c.mlp.record || c.mlp.seed_mode == SPH_SEED_MLP))
        CK(cudaMemcpyAsync(c.mlp.seed0, c.h_seed, bytes, cudaMemcpyDeviceToDevice, s));
    if (timed) CK(record(c, c.kev[0], s));
    CK(launch_walk(c, *p, WALK_DENSITY, -1, c.h_seed, s));
    if (fg) CK(launch_fastgas_mark(c, *fg, s));
    if (timed) CK(record(c, c.kev[1], s));
    CK(launch_density(c, *p, c.h_seed, -1, 0, 0, nullptr, nullptr, s, fg != nullptr));
    if (timed) CK(record(c, c.kev[2], s));
    // groups whose h left the list coverage: re-walk and re-solve on the
    // device (the launches exit at once when nothing is queued)
    for (int r = 0; r < kRelistRounds; ++r) {
        CK(launch_walk(c, *p, WALK_DENSITY, r, c.h_seed, s));
        CK(launch_density(c, *p, c.h_seed, r, 0, 0, nullptr, nullptr, s));
    }
    // evolved density: the context's first density pass starts it from the
    // kernel sum
    if (c.kp.evolved && !c.rho_evolved_init) {
        CK(cudaMemcpyAsync(p->rho, c.rho_sum, bytes, cudaMemcpyDeviceToDevice, s));
        c.rho_evolved_init = true;
    }
    CK(record(c, c.out_dens, s));  // rho, Omega, n_i, iterations are final
    CK(wait_late_inputs(c, s));  // everything before read x, m, h (and rho, id) only
    if (c.mlp.record) CK(launch_mlp_harvest(c, *p, s));
    if (isen) CK(launch_isentropic(c, *p, s));
    CK(launch_bob_refit(c, *p, s));
    return SPH_OK;
}

// fastgas: walk and sum only the marked groups (the queue q_density left)
sph_status q_forces(Ctx &c, sph_particles *p, cudaStream_t s, bool timed,
                    const RungArgs *ra = nullptr, bool fastgas = false)
{
    if (timed) CK(record(c, c.kev[3], s));
    if (c.kp.ic) {
        // interface correction (Sec. 2.3.4): predictor, then the correction
        // pass over the density lists, before the force walk replaces them
        CK(launch_predict(c, *p, s, ra));
        CK(launch_interface(c, *p, s));
        if (fastgas) CK(launch_walk_queue(c, WALK_FORCE, c.fg_list, &c.st->fg_cnt, nullptr, s));
        else CK(launch_walk(c, *p, WALK_FORCE, -1, nullptr, s));
    } else {
        // predictor + EOS on the side stream while the force walk runs here
        CK(cudaEventRecord(c.fork, s));
        CK(cudaStreamWaitEvent(c.side, c.fork, 0));
        CK(launch_predict(c, *p, c.side, ra));
        CK(cudaEventRecord(c.join, c.side));
        if (fastgas) CK(launch_walk_queue(c, WALK_FORCE, c.fg_list, &c.st->fg_cnt, nullptr, s));
        else CK(launch_walk(c, *p, WALK_FORCE, -1, nullptr, s));
        CK(cudaStreamWaitEvent(s, c.join, 0));
    }
    if (timed) CK(record(c, c.kev[4], s));
    CK(launch_forces(c, *p, s, ra, fastgas));
    if (timed) CK(record(c, c.kev[5], s));
    CK(launch_finalize(c, *p, s, ra));
    CK(record(c, c.out_force, s));  // a, du/dt, div v, dt_i are final
    return SPH_OK;
}

void density_stats(Ctx &c)
{
    const DevStatus &h = *c.st_host;
    c.stats.density_pairs = h.density_pairs;
    c.stats.density_candidates = h.density_cand;
    c.stats.max_newton_iters = h.max_iters;
    c.stats.relists = (int)(h.redo_cnt[0] + h.redo_cnt[1] + h.redo_cnt[2]);
}

void force_stats(Ctx &c)
{
    const DevStatus &h = *c.st_host;
    c.stats.force_pairs = h.force_pairs;
    c.stats.force_candidates = h.force_cand;
    c.stats.force_av_pairs = h.force_av_pairs;
}

sph_status create_ctx(const sph_params *prm, int ninst, const std::vector<int64_t> &counts,
                      int64_t capacity, sph_ctx **out)
{
    for (int k = 0; k < ninst; ++k)
        if (!params_ok(&prm[k])) return SPH_ERR_ARG;
    for (int k = 1; k < ninst; ++k)
        if (prm[k].kernel != prm[0].kernel || prm[k].energy_mode != prm[0].energy_mode ||
            prm[k].max_newton != prm[0].max_newton || prm[k].h_rel_tol != prm[0].h_rel_tol ||
            prm[k].list_margin != prm[0].list_margin || prm[k].precision != prm[0].precision ||
            prm[k].density_mode != prm[0].density_mode ||
            prm[k].interface_correction != prm[0].interface_correction)
            return SPH_ERR_ARG;
    sph_ctx *ctx = new (std::nothrow) sph_ctx;
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    c.prm.assign(prm, prm + ninst);
    c.capacity = capacity;
    c.dt_host.assign(ninst, 0.0);
    cudaGetDevice(&c.device);
    std::memset(&c.kp, 0, sizeof c.kp);
    c.kp.kernel = prm[0].kernel;
    c.kp.energy_mode = prm[0].energy_mode;
    c.kp.max_newton = prm[0].max_newton;
    c.kp.h_rel_tol = (float)prm[0].h_rel_tol;
    c.kp.h_step_tol = (float)std::min(std::sqrt(prm[0].h_rel_tol), 1e-2);
    c.kp.margin = (float)prm[0].list_margin;
    c.kp.fp64 = prm[0].precision == SPH_PRECISION_FP64 ? 1 : 0;
    c.kp.evolved = prm[0].density_mode == SPH_DENSITY_EVOLVED ? 1 : 0;
    c.kp.ic = prm[0].interface_correction;
    c.resort_period = prm[0].resort_period > 0 ? prm[0].resort_period : 1;
    c.kp.ninst = ninst;
    const Sizes z = layout_sizes(counts, c.prm);
    c.cap_nb = z.nb;
    c.cap_ng = z.ng;
    sph_status rc = allocate(c, z, ninst);
    if (rc == SPH_OK) rc = set_layout(c, counts);
    if (rc == SPH_OK && cudaDeviceSynchronize() != cudaSuccess) rc = SPH_ERR_CUDA;
    if (rc != SPH_OK) {
        free_ctx(c);
        delete ctx;
        return rc;
    }
    *out = ctx;
    return SPH_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" sph_status sph_create(const sph_params *prm, int64_t capacity, sph_ctx **out)
{
    if (!prm || !out || capacity < 0 || capacity > (int64_t)0x7fffffff - 64) return SPH_ERR_ARG;
    *out = nullptr;
    return create_ctx(prm, 1, {capacity}, capacity, out);
}

extern "C" sph_status sph_batch_create(const sph_params *params, int32_t ninst,
                                       const int64_t *offsets, sph_ctx **out)
{
    if (!params || !offsets || !out || ninst < 1 || ninst > 65535) return SPH_ERR_ARG;
    *out = nullptr;
    std::vector<int64_t> counts(ninst);
    if (offsets[0] != 0) return SPH_ERR_ARG;
    for (int k = 0; k < ninst; ++k) {
        counts[k] = offsets[k + 1] - offsets[k];
        if (counts[k] < 0) return SPH_ERR_ARG;
    }
    if (offsets[ninst] > (int64_t)0x7fffffff - 64) return SPH_ERR_ARG;
    return create_ctx(params, ninst, counts, offsets[ninst], out);
}

extern "C" void sph_destroy(sph_ctx *ctx)
{
    if (!ctx) return;
    cudaDeviceSynchronize();
    free_ctx(ctx->c);
    delete ctx;
}

extern "C" sph_status sph_build_cells(sph_ctx *ctx, sph_particles *p, void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    sph_status rc = ensure_layout(c, p);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    c.cells_valid = c.density_valid = c.forces_valid = false;
    if (p->n == 0) {
        c.cells_valid = true;
        return SPH_OK;
    }
    rc = begin(ctx, s);
    if (rc) return rc;
    CK(cudaEventRecord(c.ev0, s));
    CK(launch_build(c, *p, s));
    rc = finish(ctx, s);
    c.stats.ms_build = elapsed(c.ev0, c.ev1);
    if (rc == SPH_OK) c.cells_valid = true;
    c.order_fresh = rc == SPH_OK;
    c.since_sort = 0;
    return rc;
}

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
    sph_status rc = begin(ctx, s);
    if (rc) return rc;
    CK(cudaEventRecord(c.ev0, s));
    rc = q_density(c, p, h_seed, s, true);
    if (rc) return rc;
    rc = finish(ctx, s);
    c.stats.ms_density = elapsed(c.ev0, c.ev1);
    c.stats.ms_walk = elapsed(c.kev[0], c.kev[1]);
    c.stats.ms_density_kernel = elapsed(c.kev[1], c.kev[2]);
    density_stats(c);
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
    sph_status rc = begin(ctx, s);
    if (rc) return rc;
    CK(cudaEventRecord(c.ev0, s));
    CK(cudaMemcpyAsync(c.h_seed, h, sizeof(float) * (size_t)p->n, cudaMemcpyDeviceToDevice, s));
    CK(launch_walk(c, *p, WALK_DENSITY, -1, c.h_seed, s));
    CK(launch_density(c, *p, c.h_seed, -1, 1, cap, count, ids, s));
    rc = finish(ctx, s);
    c.density_valid = false;
    c.forces_valid = false;
    return rc;
}

extern "C" sph_status sph_forces(sph_ctx *ctx, sph_particles *p, void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (!particles_ok(p)) return failf(c, SPH_ERR_ARG, "sph_forces: NULL array");
    if (c.kp.ic && p->n > 0 && !p->mat)
        return failf(c, SPH_ERR_ARG, "the interface correction needs material ids (p->mat)");
    if (!c.density_valid || p->n != c.n_built)
        return failf(c, SPH_ERR_STATE, "sph_forces needs sph_density_h on these particles first");
    if (p->n == 0) {
        c.forces_valid = true;
        return SPH_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    sph_status rc = begin(ctx, s);
    if (rc) return rc;
    CK(cudaEventRecord(c.ev0, s));
    rc = q_forces(c, p, s, true);
    if (rc) return rc;
    rc = finish(ctx, s);
    c.stats.ms_forces = elapsed(c.ev0, c.ev1);
    c.stats.ms_walk += elapsed(c.kev[3], c.kev[4]);
    c.stats.ms_force_kernel = elapsed(c.kev[4], c.kev[5]);
    force_stats(c);
    if (rc == SPH_OK) c.forces_valid = true;
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
    CK(cudaEventRecord(c.ev0, s));
    CK(launch_kdk(c, *p, dt_fixed, s));
    rc = finish(ctx, s);
    c.stats.ms_kdk = elapsed(c.ev0, c.ev1);
    c.cells_valid = c.density_valid = c.forces_valid = false;
    if (rc == SPH_OK) {
        for (int k = 0; k < c.kp.ninst; ++k) c.dt_host[k] = c.dts_host[2 * k];
        c.stats.dt_old = c.dt_host[0];
        if (dt_used) *dt_used = c.dt_host[0];
    }
    return rc;
}

namespace {
// does the next sph_step / replay re-sort (else it refits the buckets)?
bool need_full_build(const Ctx &c)
{
    return !c.order_fresh || c.since_sort + 1 >= c.resort_period;
}

void count_build(Ctx &c, bool full, sph_status rc)
{
    if (rc != SPH_OK) {
        c.order_fresh = false;
    } else if (full) {
        c.order_fresh = true;
        c.since_sort = 0;
    } else {
        ++c.since_sort;
    }
}

// the whole step queued without host round trips
sph_status queue_step(Ctx &c, sph_particles *p, double dt_fixed, cudaStream_t s, bool timed,
                      bool full_build)
{
    if (timed) CK(record(c, c.ev0, s));
    if (full_build) {
        CK(wait_late_inputs(c, s));  // the re-sort permutes every array
        CK(launch_build(c, *p, s));
    } else {
        CK(launch_refit(c, *p, s));
    }
    sph_status rc = q_density(c, p, nullptr, s, timed);
    if (rc) return rc;
    rc = q_forces(c, p, s, timed);
    if (rc) return rc;
    CK(launch_kdk(c, *p, dt_fixed, s));
    return SPH_OK;
}

void step_done(Ctx &c, sph_status rc, bool timed)
{
    if (timed) {
        c.stats.ms_build = elapsed(c.ev0, c.kev[0]);
        c.stats.ms_walk = elapsed(c.kev[0], c.kev[1]) + elapsed(c.kev[3], c.kev[4]);
        c.stats.ms_density_kernel = elapsed(c.kev[1], c.kev[2]);
        c.stats.ms_force_kernel = elapsed(c.kev[4], c.kev[5]);
        c.stats.ms_density = elapsed(c.kev[0], c.kev[3]);
        c.stats.ms_forces = elapsed(c.kev[3], c.ev1);
    }
    density_stats(c);
    force_stats(c);
    c.cells_valid = c.density_valid = c.forces_valid = false;
    if (rc == SPH_OK) {
        c.rho_valid = true;
        for (int k = 0; k < c.kp.ninst; ++k) c.dt_host[k] = c.dts_host[2 * k];
        c.stats.dt_old = c.dt_host[0];
    }
}
}  // namespace

extern "C" sph_status sph_step(sph_ctx *ctx, sph_particles *p, double dt_fixed, double *dt_used,
                               void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    sph_status rc = ensure_layout(c, p);
    if (rc) return rc;
    if (!(dt_fixed == dt_fixed) || std::isinf(dt_fixed))
        return failf(c, SPH_ERR_ARG, "sph_step: dt_fixed must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    if (p->n == 0) {
        if (dt_used) *dt_used = dt_fixed > 0 ? dt_fixed : 0.0;
        return SPH_OK;
    }
    rc = begin(ctx, s);
    if (rc) return rc;
    const bool full = need_full_build(c);
    rc = queue_step(c, p, dt_fixed, s, true, full);
    if (rc) return rc;
    rc = finish(ctx, s);
    step_done(c, rc, true);
    count_build(c, full, rc);
    if (rc == SPH_OK && dt_used) *dt_used = c.dt_host[0];
    return rc;
}

extern "C" sph_status sph_step_rungs(sph_ctx *ctx, sph_particles *p, double dt0, int32_t max_rung,
                                     void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    sph_status rc = ensure_layout(c, p);
    if (rc) return rc;
    if (!(dt0 > 0.0) || std::isinf(dt0))
        return failf(c, SPH_ERR_ARG, "sph_step_rungs: dt0 must be positive and finite");
    if (max_rung < 0 || max_rung > 20)
        return failf(c, SPH_ERR_ARG, "sph_step_rungs: max_rung must be in [0, 20]");
    if (c.kp.fp64 || c.kp.evolved)
        return failf(c, SPH_ERR_ARG, "sph_step_rungs: mixed precision and summed density only");
    if (c.mlp.record || c.mlp.seed_mode != SPH_SEED_ANALYTIC)
        return failf(c, SPH_ERR_STATE, "sph_step_rungs: the learned seed is for global steps");
    if (!c.rungs_started && c.dt_host[0] > 0.0)
        return failf(c, SPH_ERR_STATE, "hierarchical steps continue only a run begun with them "
                     "(sph_set_dt_old(ctx, 0) restarts)");
    if (c.rungs_started && max_rung != c.rung_R)
        return failf(c, SPH_ERR_STATE, "sph_step_rungs: max_rung must stay %d", c.rung_R);
    if (p->n == 0) return SPH_OK;
    const size_t cap = (size_t)(c.capacity > 0 ? c.capacity : 1);
    if (!c.rung) {
        if (dalloc(&c.rung, cap) != cudaSuccess || dalloc(&c.rmax, cap) != cudaSuccess)
            return failf(c, SPH_ERR_CUDA, "cudaMalloc of the rung arrays failed");
        CK(cudaMemset(c.rung, 0, cap));
    }
    if (c.fastgas && !c.bact) {
        const size_t nbc = (size_t)std::max<int64_t>(c.cap_nb, 1);
        const size_t ngc = (size_t)std::max<int64_t>(c.cap_ng, 1);
        if (dalloc(&c.bact, nbc) != cudaSuccess || dalloc(&c.gmark, ngc) != cudaSuccess ||
            dalloc(&c.fg_list, ngc) != cudaSuccess)
            return failf(c, SPH_ERR_CUDA, "cudaMalloc of the FastGas arrays failed");
    }
    cudaStream_t s = (cudaStream_t)stream;
    rc = begin(ctx, s);
    if (rc) return rc;
    CK(cudaEventRecord(c.ev0, s));
    const int nsub = 1 << max_rung;
    RungArgs ra{c.rung, c.rmax, 0, max_rung, c.rungs_started ? 1 : 0, dt0 / nsub, dt0};
    for (int sub = 0; sub < nsub && rc == SPH_OK; ++sub) {
        ra.sub = sub;
        // the first substep re-sorts (the rungs move with the particles), the
        // others refit the bounds to the drifted particles
        if (sub == 0) CK(launch_build(c, *p, s));
        else CK(launch_refit(c, *p, s));
        rc = q_density(c, p, nullptr, s, false, c.fastgas ? &ra : nullptr);
        if (rc == SPH_OK) rc = q_forces(c, p, s, false, &ra, c.fastgas);
        if (rc == SPH_OK) CK(launch_kdk_rungs(c, *p, ra, s));
        ra.started = 1;
    }
    if (rc) return rc;
    rc = finish(ctx, s);
    c.stats.ms_forces = elapsed(c.ev0, c.ev1);
    density_stats(c);
    force_stats(c);
    c.cells_valid = c.density_valid = c.forces_valid = false;
    c.order_fresh = false;
    if (rc == SPH_OK) {
        c.rungs_started = true;
        c.rung_R = max_rung;
        c.rho_valid = true;
    }
    return rc;
}

extern "C" sph_status sph_set_fastgas(sph_ctx *ctx, int32_t on)
{
    if (!ctx) return SPH_ERR_ARG;
    ctx->c.fastgas = on != 0;
    return SPH_OK;
}

extern "C" sph_status sph_get_rungs(sph_ctx *ctx, uint8_t *out, int64_t n)
{
    if (!ctx || !out || n < 0) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (n > c.n_built) return failf(c, SPH_ERR_ARG, "n exceeds the particles of the context");
    if (!c.rung) {
        std::memset(out, 0, (size_t)n);
        return SPH_OK;
    }
    CK(cudaMemcpy(out, c.rung, (size_t)n, cudaMemcpyDeviceToHost));
    return SPH_OK;
}

namespace {
sph_status capture_step(Ctx &c, sph_particles *p, double dt_fixed, cudaStream_t s, bool full);
}

extern "C" sph_status sph_graph_capture(sph_ctx *ctx, sph_particles *p, double dt_fixed,
                                        void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    sph_status rc = ensure_layout(c, p);
    if (rc) return rc;
    if (!stream) return failf(c, SPH_ERR_ARG, "sph_graph_capture needs a non-default stream");
    if (p->n == 0) return failf(c, SPH_ERR_ARG, "sph_graph_capture needs particles");
    if (!(dt_fixed == dt_fixed) || std::isinf(dt_fixed))
        return failf(c, SPH_ERR_ARG, "sph_graph_capture: dt_fixed must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    for (cudaGraphExec_t *ge : {&c.graph_exec, &c.graph_exec_r})
        if (*ge) cudaGraphExecDestroy(*ge);
    for (cudaGraph_t *gr : {&c.graph, &c.graph_r})
        if (*gr) cudaGraphDestroy(*gr);
    c.graph_exec = c.graph_exec_r = nullptr;
    c.graph = c.graph_r = nullptr;
    c.graph_replayed = false;
    // one graph that re-sorts, and with a re-sort period one that refits
    for (int mode = 0; mode < (c.resort_period > 1 ? 2 : 1); ++mode) {
        const sph_status r = capture_step(c, p, dt_fixed, s, mode == 0);
        if (r) return r;
    }
    c.graph_p = *p;
    c.graph_dt = dt_fixed;
    return SPH_OK;
}

namespace {
sph_status capture_step(Ctx &c, sph_particles *p, double dt_fixed, cudaStream_t s, bool full)
{
    // the start of the evolved density is a one-off copy, not part of a step
    if (c.kp.evolved && !c.rho_evolved_init)
        return failf(c, SPH_ERR_STATE, "evolved density: step once before recording a step");
    const uint64_t l0 = c.launches;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    c.err.clear();
    c.capturing = true;
    sph_status qrc = SPH_OK;
    c.prof.slot = full ? 0 : 1;
    c.prof.gphase[c.prof.slot].clear();
    if (cudaMemsetAsync(c.st, 0, sizeof(DevStatus), s) != cudaSuccess) qrc = SPH_ERR_CUDA;
    // phase events are captured too (event record nodes), so a replay reports
    // the same per-phase times as sph_step (and, with profiling on while
    // capturing, the same launch groups)
    if (qrc == SPH_OK) qrc = queue_step(c, p, dt_fixed, s, true, full);
    // the totals of the stepped state ride along (read with sph_graph_totals)
    if (qrc == SPH_OK && launch_conserved(c, *p, s) != cudaSuccess) qrc = SPH_ERR_CUDA;
    if (qrc == SPH_OK && cudaMemcpyAsync(c.cons_host, c.cons_out, sizeof(double) * 9 * c.kp.ninst,
                                         cudaMemcpyDeviceToHost, s) != cudaSuccess)
        qrc = SPH_ERR_CUDA;
    if (qrc == SPH_OK) qrc = queue_status(c, s);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    c.capturing = false;
    const uint64_t kernels = c.launches - l0;
    c.launches = l0;
    if (qrc != SPH_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        return failf(c, SPH_ERR_CUDA, "stream capture of the step failed: %s",
                     e != cudaSuccess ? cudaGetErrorString(e) : c.err.c_str());
    }
    if (full) {
        c.graph = g;
        CK(cudaGraphInstantiate(&c.graph_exec, g, 0));
        c.graph_kernels = kernels;
    } else {
        c.graph_r = g;
        CK(cudaGraphInstantiate(&c.graph_exec_r, g, 0));
        c.graph_kernels_r = kernels;
    }
    return SPH_OK;
}
}  // namespace

extern "C" sph_status sph_graph_totals(const sph_ctx *ctx, double *out)
{
    if (!ctx || !out) return SPH_ERR_ARG;
    const Ctx &c = ctx->c;
    if (!c.graph_exec || !c.graph_replayed) return SPH_ERR_STATE;
    std::memcpy(out, c.graph_totals.data(), sizeof(double) * c.graph_totals.size());
    return SPH_OK;
}

namespace {
// replay of the captured step, queued only (the re-sorting graph when a
// re-sort is due)
sph_status graph_enqueue(Ctx &c, cudaStream_t s, bool *full)
{
    c.err.clear();
    *full = need_full_build(c) || !c.graph_exec_r;
    CK(cudaGraphLaunch(*full ? c.graph_exec : c.graph_exec_r, s));
    CK(cudaEventRecord(c.ev1, s));
    c.launches += *full ? c.graph_kernels : c.graph_kernels_r;
    return SPH_OK;
}

// wait for a queued replay and take its status, step size and totals
sph_status graph_settle(sph_ctx *ctx, cudaStream_t s, bool full, double *dt_used)
{
    Ctx &c = ctx->c;
    sph_status rc = settle(ctx, s);
    if (rc == SPH_OK && c.prof.on) prof_collect_graph(c, full ? 0 : 1);
    step_done(c, rc, true);
    count_build(c, full, rc);
    if (rc == SPH_OK) {
        c.graph_totals.assign(c.cons_host, c.cons_host + 9 * c.kp.ninst);
        c.graph_replayed = true;
    }
    if (rc == SPH_OK && dt_used) *dt_used = c.dt_host[0];
    return rc;
}
}  // namespace

extern "C" sph_status sph_graph_launch(sph_ctx *ctx, double *dt_used, void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (!c.graph_exec) return failf(c, SPH_ERR_STATE, "no captured step: call sph_graph_capture");
    cudaStream_t s = (cudaStream_t)stream;
    bool full = false;
    sph_status rc = graph_enqueue(c, s, &full);
    if (rc) return rc;
    return graph_settle(ctx, s, full, dt_used);
}

namespace {
struct ArrDesc {
    size_t off;   // offset of the pointer member in sph_particles
    size_t elem;  // element size
    int in;       // read by a step: 1 always, 2 in SPH_ENERGY_ISENTROPIC mode or with the
                  // evolved density, 3 with the evolved density, 4 with the interface
                  // correction (and copied back only then), 0 never
    int late;     // first read after the density phase (1): copied in beside the step
    int out;      // final after the density phase (1), after the forces (2), at the end (0)
    int sorted;   // changed only by a re-sort (1: m, id), so unchanged by a refitting step
    int sort_in;  // read only by a re-sort (1: id)
};
const ArrDesc kArrays[] = {
    {offsetof(sph_particles, x) + 0 * sizeof(double *), 8, 1, 0, 0, 0, 0},
    {offsetof(sph_particles, x) + 1 * sizeof(double *), 8, 1, 0, 0, 0, 0},
    {offsetof(sph_particles, x) + 2 * sizeof(double *), 8, 1, 0, 0, 0, 0},
    {offsetof(sph_particles, v) + 0 * sizeof(double *), 8, 1, 1, 0, 0, 0},
    {offsetof(sph_particles, v) + 1 * sizeof(double *), 8, 1, 1, 0, 0, 0},
    {offsetof(sph_particles, v) + 2 * sizeof(double *), 8, 1, 1, 0, 0, 0},
    {offsetof(sph_particles, u), 8, 1, 1, 0, 0, 0},
    {offsetof(sph_particles, m), 4, 1, 0, 0, 1, 0},
    {offsetof(sph_particles, h), 4, 1, 0, 0, 0, 0},
    {offsetof(sph_particles, rho), 4, 2, 0, 1, 0, 0},
    {offsetof(sph_particles, omega), 4, 0, 0, 1, 0, 0},
    {offsetof(sph_particles, a) + 0 * sizeof(float *), 4, 1, 1, 2, 0, 0},
    {offsetof(sph_particles, a) + 1 * sizeof(float *), 4, 1, 1, 2, 0, 0},
    {offsetof(sph_particles, a) + 2 * sizeof(float *), 4, 1, 1, 2, 0, 0},
    {offsetof(sph_particles, dudt_h), 4, 1, 1, 2, 0, 0},
    {offsetof(sph_particles, dudt_av), 4, 1, 1, 2, 0, 0},
    {offsetof(sph_particles, divv), 4, 3, 1, 2, 0, 0},
    {offsetof(sph_particles, dt_i), 4, 0, 0, 2, 0, 0},
    {offsetof(sph_particles, nngb), 2, 0, 0, 1, 0, 0},
    {offsetof(sph_particles, iters), 1, 0, 0, 1, 0, 0},
    {offsetof(sph_particles, id), 8, 1, 0, 0, 1, 1},
    {offsetof(sph_particles, mat), 1, 4, 0, 0, 1, 0},
};
void *&member(sph_particles &p, const ArrDesc &d)
{
    return *reinterpret_cast<void **>(reinterpret_cast<char *>(&p) + d.off);
}
}  // namespace

namespace {
// Host <-> device copies of sph_step_host.  Host arrays the GPU can address
// (pinned memory, mapped into the device's address space) are moved by ONE
// kernel per direction that reads or writes them over the CPU-GPU link,
// every array in the same launch: per-array copy-engine transfers cost a few
// microseconds each, which for the 15 input (16 in the entropy-conserving
// mode) and 21 output arrays of a step is more than the data time.  Other host memory (pageable) goes through
// cudaMemcpyAsync.
constexpr int kMaxCopy = sizeof(kArrays) / sizeof(kArrays[0]);
struct CopyJob {
    const char *src[kMaxCopy];
    char *dst[kMaxCopy];
    unsigned long long bytes[kMaxCopy];
};

// blockIdx.y = array; 16-byte words where both ends are 16-byte aligned, the
// ragged tail (or a misaligned array) byte by byte
__global__ void __launch_bounds__(256) k_copy_arrays(CopyJob job)
{
    const int a = blockIdx.y;
    const char *__restrict__ src = job.src[a];
    char *__restrict__ dst = job.dst[a];
    const unsigned long long nb = job.bytes[a];
    const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned long long done = 0;
    if ((((uintptr_t)src | (uintptr_t)dst) & 15u) == 0) {
        const unsigned long long n16 = nb / 16;
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
        for (unsigned long long i = t; i < n16; i += stride) d4[i] = s4[i];
        done = n16 * 16;
    }
    for (unsigned long long i = done + t; i < nb; i += stride) dst[i] = src[i];
}

// device address of each host array (NULL where the GPU cannot address it),
// looked up on every call: an address the caller freed and reused for
// pageable memory must not keep an old mapping
void map_host(Ctx &c, const sph_host_particles *hp)
{
    c.hkey = *hp;
    for (const ArrDesc &d : kArrays) {
        void *h = member(c.hkey, d);
        void *dev = nullptr;
        cudaPointerAttributes at;
        if (h && cudaPointerGetAttributes(&at, h) == cudaSuccess && at.type == cudaMemoryTypeHost)
            dev = at.devicePointer;
        cudaGetLastError();  // a failed lookup only means "not mapped"
        member(c.hdev, d) = dev;
    }
}

// copy n elements of every selected array, host -> mirror (in) or mirror ->
// host (!in).  part 0: all; in: 1 the arrays read early in a step, 2 the late
// ones (ArrDesc::late); out: 1 the density outputs, 2 the force outputs, 3
// the rest (ArrDesc::out).  engines: copy-engine transfers only (no SMs
// taken from kernels running beside them).  skip_sorted: leave out the
// arrays only a re-sort reads (in) or changes (out).  Returns the bytes
// moved.
cudaError_t copy_arrays(Ctx &c, const sph_host_particles *hp, bool in, cudaStream_t s,
                        int64_t *moved, int part = 0, bool engines = false,
                        bool skip_sorted = false)
{
    const bool isen = c.kp.energy_mode == SPH_ENERGY_ISENTROPIC;
    const bool evo = c.kp.evolved != 0;
    CopyJob job;
    int na = 0;
    unsigned long long most = 0;
    int64_t b_all = 0;
    for (const ArrDesc &d : kArrays) {
        if (in && (d.in == 0 || (d.in == 2 && !isen && !evo) || (d.in == 3 && !evo))) continue;
        if (d.in == 4 && !c.kp.ic) continue;  // material ids only matter to the correction
        if (in && ((part == 1 && d.late) || (part == 2 && !d.late))) continue;
        if (!in && part > 0 && d.out != part % 3) continue;
        if (skip_sorted && (in ? d.sort_in : d.sorted)) continue;
        const size_t b = d.elem * (size_t)hp->n;
        if (b == 0) continue;
        b_all += (int64_t)b;
        char *host = (char *)member(*const_cast<sph_host_particles *>(hp), d);
        char *mapped = engines ? nullptr : (char *)member(c.hdev, d);
        char *dev = (char *)member(c.dmirror, d);
        if (mapped) {
            job.src[na] = in ? mapped : dev;
            job.dst[na] = in ? dev : mapped;
            job.bytes[na] = b;
            most = std::max<unsigned long long>(most, b);
            ++na;
        } else {
            cudaError_t e = cudaMemcpyAsync(in ? dev : host, in ? host : dev, b,
                                            in ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost,
                                            s);
            if (e != cudaSuccess) return e;
        }
    }
    if (na > 0) {
        // about four blocks per SM over all arrays, at most one 16-byte word
        // per thread of the largest array
        const unsigned long long words = (most + 15) / 16;
        unsigned gx = (unsigned)std::min<unsigned long long>(
            (words + 255) / 256, (unsigned long long)std::max(1, 608 / na));
        c.launches += 1;
        k_copy_arrays<<<dim3(std::max(gx, 1u), (unsigned)na), 256, 0, s>>>(job);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (moved) *moved = b_all;
    return cudaSuccess;
}

// device mirror of the host arrays (allocated once for the capacity) and the
// host-to-device copy of the arrays a step reads
sph_status host_in(Ctx &c, const sph_host_particles *hp, cudaStream_t s, int64_t *moved,
                   bool refit_replay = false)
{
    const size_t cap = (size_t)(c.capacity > 0 ? c.capacity : 1);
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
    map_host(c, hp);
    // the early inputs first, with the whole link; then the late ones on
    // the copy stream by the copy engines, beside the first phases of the
    // step (refit, walk, density), which wait for them only at their end
    int64_t b1 = 0, b2 = 0;
    CK(copy_arrays(c, hp, true, s, &b1, 1, false, refit_replay));
    CK(cudaEventRecord(c.call0, s));
    CK(cudaStreamWaitEvent(c.copy, c.call0, 0));
    CK(copy_arrays(c, hp, true, c.copy, &b2, 2, true));
    CK(cudaEventRecord(c.late_in, c.copy));
    if (moved) *moved = b1 + b2;
    return SPH_OK;
}

bool graph_on_mirror(const Ctx &c, double dt_fixed)
{
    if (!c.graph_exec || !c.mirror || c.graph_dt != dt_fixed) return false;
    if (c.graph_p.n != c.dmirror.n) return false;
    for (const ArrDesc &d : kArrays)
        if (member(const_cast<sph_particles &>(c.graph_p), d) !=
            member(const_cast<sph_particles &>(c.dmirror), d))
            return false;
    return true;
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
    int64_t moved = 0;
    // a replay of the recorded step that only refits reads no id (only a
    // re-sort permutes it): the mirror's copy is refreshed by the next
    // re-sorting step's input copy, and the host's stays as it is
    const bool replay = c.mirror && hp->n == c.dmirror.n && graph_on_mirror(c, dt_fixed);
    const bool refit_replay = replay && !(need_full_build(c) || !c.graph_exec_r);
    sph_status rc = host_in(c, hp, s, &moved, refit_replay);
    if (rc) return rc;
    if (h2d_bytes) *h2d_bytes = moved;
    int64_t out = 0;
    if (graph_on_mirror(c, dt_fixed)) {
        // the step sph_step_host_capture recorded for these buffers and this
        // dt_fixed.  Outputs that are final before the step ends are copied
        // back by the copy engines while it finishes (the replay records
        // the events out_dens and out_force at those points), the rest by
        // the copy kernel after it; one wait for all.  On an error status
        // the host arrays hold what the failed step left in the device
        // buffers (x, v, u as they were).
        bool full = false;
        rc = graph_enqueue(c, s, &full);
        if (rc) return rc;
        int64_t o1 = 0, o2 = 0, o3 = 0;
        CK(cudaStreamWaitEvent(c.copy, c.out_dens, 0));
        CK(copy_arrays(c, hp, false, c.copy, &o1, 1, true));
        CK(cudaStreamWaitEvent(c.copy, c.out_force, 0));
        CK(copy_arrays(c, hp, false, c.copy, &o2, 2, true));
        CK(cudaEventRecord(c.out_done, c.copy));
        // a refitting replay leaves m and id as they were copied in: the
        // host arrays already hold them
        CK(copy_arrays(c, hp, false, s, &o3, 3, false, !full));
        CK(cudaStreamWaitEvent(s, c.out_done, 0));
        out = o1 + o2 + o3;
        rc = graph_settle(ctx, s, full, dt_used);
        if (rc) return rc;
    } else {
        rc = sph_step(ctx, &c.dmirror, dt_fixed, dt_used, stream);
        if (rc) return rc;
        CK(copy_arrays(c, hp, false, s, &out));
        CK(cudaStreamSynchronize(s));
    }
    if (d2h_bytes) *d2h_bytes = out;
    return SPH_OK;
}

extern "C" sph_status sph_step_host_capture(sph_ctx *ctx, sph_host_particles *hp,
                                            double dt_fixed, void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (!particles_ok(hp) || hp->n > c.capacity)
        return failf(c, SPH_ERR_ARG, "sph_step_host_capture: NULL array or n > capacity");
    cudaStream_t s = (cudaStream_t)stream;
    sph_status rc = host_in(c, hp, s, nullptr);
    if (rc) return rc;
    CK(cudaStreamSynchronize(s));
    CK(cudaStreamSynchronize(c.copy));
    return sph_graph_capture(ctx, &c.dmirror, dt_fixed, stream);
}

extern "C" sph_status sph_reduce_conserved(sph_ctx *ctx, const sph_particles *p, double *out,
                                           void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (!particles_ok(p) || !out) return failf(c, SPH_ERR_ARG, "sph_reduce_conserved: bad arguments");
    sph_status rc = ensure_layout(c, p);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = begin(ctx, s);
    if (rc) return rc;
    CK(cudaEventRecord(c.ev0, s));
    CK(launch_conserved(c, *p, s));
    CK(cudaMemcpyAsync(c.cons_host, c.cons_out, sizeof(double) * 9 * c.kp.ninst,
                       cudaMemcpyDeviceToHost, s));
    rc = finish(ctx, s);
    if (rc == SPH_OK) std::memcpy(out, c.cons_host, sizeof(double) * 9 * c.kp.ninst);
    return rc;
}

// ---- learned seed -------------------------------------------------------------
namespace {
// network buffers (zero weights = the continuity estimate) on first use
sph_status ensure_mlp(Ctx &c)
{
    if (c.mlp.w) return SPH_OK;
    CK(dalloc(&c.mlp.w, kMlpParams));
    CK(dalloc(&c.mlp.m, kMlpParams));
    CK(dalloc(&c.mlp.v, kMlpParams));
    CK(dalloc(&c.mlp.frag, kMlpFragWords));
    CK(dalloc(&c.mlp.scount, 1));
    CK(dalloc(&c.mlp.seed0, (size_t)std::max<int64_t>(c.capacity, 1)));
    CK(dalloc(&c.mlp.corr, (size_t)std::max<int64_t>(c.capacity, 1)));
    CK(cudaMemset(c.mlp.seed0, 0, sizeof(float) * (size_t)std::max<int64_t>(c.capacity, 1)));
    CK(cudaMemset(c.mlp.w, 0, sizeof(float) * kMlpParams));
    CK(cudaMemset(c.mlp.m, 0, sizeof(float) * kMlpParams));
    CK(cudaMemset(c.mlp.v, 0, sizeof(float) * kMlpParams));
    CK(cudaMemset(c.mlp.scount, 0, sizeof(unsigned long long)));
    CK(launch_mlp_pack(c, nullptr));
    CK(cudaDeviceSynchronize());
    return SPH_OK;
}

// sample buffer of at least `cap` samples (contents dropped when it grows)
sph_status ensure_samples(Ctx &c, int64_t cap)
{
    if (c.mlp.sx && c.mlp.cap >= cap) return SPH_OK;
    CK(cudaDeviceSynchronize());
    if (c.mlp.sx) cudaFree(c.mlp.sx);
    if (c.mlp.sy) cudaFree(c.mlp.sy);
    c.mlp.sx = c.mlp.sy = nullptr;
    c.mlp.cap = 0;
    CK(dalloc(&c.mlp.sx, (size_t)cap * 4));
    CK(dalloc(&c.mlp.sy, (size_t)cap));
    CK(cudaMemset(c.mlp.scount, 0, sizeof(unsigned long long)));
    c.mlp.cap = cap;
    return SPH_OK;
}

sph_status ensure_grad_space(Ctx &c, long long batch, int iters)
{
    const int nb = mlp_grad_blocks(batch);
    if (c.mlp.gpart_blocks < nb) {
        if (c.mlp.gpart) cudaFree(c.mlp.gpart);
        c.mlp.gpart = nullptr;
        c.mlp.gpart_blocks = 0;
        CK(dalloc(&c.mlp.gpart, (size_t)nb * (kMlpParams + 1)));
        c.mlp.gpart_blocks = nb;
    }
    if (c.mlp.loss_cap < iters) {
        if (c.mlp.loss) cudaFree(c.mlp.loss);
        c.mlp.loss = nullptr;
        c.mlp.loss_cap = 0;
        CK(dalloc(&c.mlp.loss, (size_t)iters));
        c.mlp.loss_cap = iters;
    }
    return SPH_OK;
}

int64_t samples_held(Ctx &c)
{
    unsigned long long cnt = 0;
    if (cudaMemcpy(&cnt, c.mlp.scount, sizeof cnt, cudaMemcpyDeviceToHost) != cudaSuccess)
        return -1;
    return (int64_t)(cnt < (unsigned long long)c.mlp.cap ? cnt : (unsigned long long)c.mlp.cap);
}
}  // namespace

extern "C" sph_status sph_mlp_set_weights(sph_ctx *ctx, const float *w, int64_t count)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (!w || count != kMlpParams)
        return failf(c, SPH_ERR_ARG, "sph_mlp_set_weights needs %d floats", kMlpParams);
    sph_status rc = ensure_mlp(c);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(c.mlp.w, w, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice));
    CK(cudaMemset(c.mlp.m, 0, sizeof(float) * kMlpParams));
    CK(cudaMemset(c.mlp.v, 0, sizeof(float) * kMlpParams));
    c.mlp.t = 0;
    c.mlp.dead = 0.f;
    CK(launch_mlp_pack(c, nullptr));
    CK(cudaDeviceSynchronize());
    return SPH_OK;
}

extern "C" sph_status sph_mlp_get_weights(sph_ctx *ctx, float *w, int64_t count)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (!w || count != kMlpParams)
        return failf(c, SPH_ERR_ARG, "sph_mlp_get_weights needs %d floats", kMlpParams);
    sph_status rc = ensure_mlp(c);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(w, c.mlp.w, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
    return SPH_OK;
}

extern "C" sph_status sph_mlp_set_seed_mode(sph_ctx *ctx, int32_t mode)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (mode != SPH_SEED_ANALYTIC && mode != SPH_SEED_MLP)
        return failf(c, SPH_ERR_ARG, "unknown seed mode %d", mode);
    sph_status rc = ensure_mlp(c);
    if (rc) return rc;
    c.mlp.seed_mode = mode;
    return SPH_OK;
}

extern "C" sph_status sph_mlp_record(sph_ctx *ctx, int32_t on, int64_t capacity, int32_t stride)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (!on) {
        c.mlp.record = false;
        return SPH_OK;
    }
    if (capacity < 1 || stride < 1)
        return failf(c, SPH_ERR_ARG, "sph_mlp_record: capacity and stride must be >= 1");
    sph_status rc = ensure_mlp(c);
    if (rc) return rc;
    if (!c.mlp.th) {
        CK(dalloc(&c.mlp.tfeat, (size_t)c.capacity * 4));
        CK(dalloc(&c.mlp.th, (size_t)c.capacity));
    }
    rc = ensure_samples(c, capacity);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    CK(cudaMemset(c.mlp.th, 0, sizeof(float) * (size_t)std::max<int64_t>(c.capacity, 1)));
    c.mlp.stride = stride;
    c.mlp.record = true;
    return SPH_OK;
}

extern "C" sph_status sph_mlp_samples(sph_ctx *ctx, int64_t *count)
{
    if (!ctx || !count) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    *count = 0;
    if (!c.mlp.sx) return SPH_OK;
    CK(cudaDeviceSynchronize());
    const int64_t k = samples_held(c);
    if (k < 0) return failf(c, SPH_ERR_CUDA, "sph_mlp_samples: read-back failed");
    *count = k;
    return SPH_OK;
}

extern "C" sph_status sph_mlp_get_samples(sph_ctx *ctx, float *x, float *y, int64_t n)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (n < 0 || (n > 0 && (!x || !y))) return failf(c, SPH_ERR_ARG, "sph_mlp_get_samples");
    if (n == 0) return SPH_OK;
    if (!c.mlp.sx) return failf(c, SPH_ERR_ARG, "sph_mlp_get_samples: no samples");
    CK(cudaDeviceSynchronize());
    if (n > samples_held(c))
        return failf(c, SPH_ERR_ARG, "sph_mlp_get_samples: fewer than %lld samples", (long long)n);
    CK(cudaMemcpy(x, c.mlp.sx, sizeof(float) * 4 * (size_t)n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(y, c.mlp.sy, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost));
    return SPH_OK;
}

extern "C" sph_status sph_mlp_load_samples(sph_ctx *ctx, const float *x, const float *y,
                                           int64_t n, void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (n < 1 || !x || !y) return failf(c, SPH_ERR_ARG, "sph_mlp_load_samples: need n >= 1");
    sph_status rc = ensure_mlp(c);
    if (rc) return rc;
    rc = ensure_samples(c, n);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned long long cnt = (unsigned long long)n;
    CK(cudaMemcpyAsync(c.mlp.sx, x, sizeof(float) * 4 * (size_t)n, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c.mlp.sy, y, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c.mlp.scount, &cnt, sizeof cnt, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return SPH_OK;
}

extern "C" sph_status sph_mlp_train(sph_ctx *ctx, int32_t iters, int32_t batch, double lr,
                                    uint64_t seed, double *loss_first, double *loss_last,
                                    void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (iters < 1 || !(lr > 0.0)) return failf(c, SPH_ERR_ARG, "sph_mlp_train: iters, lr");
    sph_status rc = ensure_mlp(c);
    if (rc) return rc;
    if (!c.mlp.sx) return failf(c, SPH_ERR_STATE, "sph_mlp_train: no samples");
    CK(cudaDeviceSynchronize());
    const int64_t count = samples_held(c);
    if (count <= 0) return failf(c, SPH_ERR_STATE, "sph_mlp_train: no samples");
    const bool random = batch > 0 && batch < count;
    const long long B = random ? batch : count;
    rc = ensure_grad_space(c, B, iters);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    for (int it = 0; it < iters; ++it) {
        CK(launch_mlp_grad(c, c.mlp.sx, c.mlp.sy, count, B, random ? 1 : 0, seed, it, s));
        CK(launch_mlp_update(c, B, 1, lr, nullptr, c.mlp.loss + it, s));
    }
    CK(launch_mlp_pack(c, s));
    CK(cudaStreamSynchronize(s));
    double l0 = 0.0, l1 = 0.0;
    CK(cudaMemcpy(&l0, c.mlp.loss, sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&l1, c.mlp.loss + iters - 1, sizeof(double), cudaMemcpyDeviceToHost));
    if (loss_first) *loss_first = l0;
    if (loss_last) *loss_last = l1;
    if (!std::isfinite(l1)) return failf(c, SPH_ERR_NONFINITE, "sph_mlp_train: loss is not finite");
    // the network's own fit error, in ln h: smaller corrections are noise
    c.mlp.dead = (float)(std::sqrt(l1) / kMlpYScale);
    return SPH_OK;
}

extern "C" sph_status sph_mlp_grad(sph_ctx *ctx, const float *x, const float *y, int64_t n,
                                   float *grad, double *loss, void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (n < 1 || !x || !y || !grad) return failf(c, SPH_ERR_ARG, "sph_mlp_grad: arguments");
    sph_status rc = ensure_mlp(c);
    if (rc) return rc;
    rc = ensure_grad_space(c, n, 1);
    if (rc) return rc;
    float *gdev = nullptr;
    CK(dalloc(&gdev, kMlpParams));
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_mlp_grad(c, x, y, n, n, 0, 0ull, 0, s);
    if (e == cudaSuccess) e = launch_mlp_update(c, n, 0, 0.0, gdev, c.mlp.loss, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess)
        e = cudaMemcpy(grad, gdev, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && loss) e = cudaMemcpy(loss, c.mlp.loss, sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(gdev);
    if (e != cudaSuccess) return failf(c, SPH_ERR_CUDA, "sph_mlp_grad: %s", cudaGetErrorString(e));
    return SPH_OK;
}

extern "C" sph_status sph_mlp_infer(sph_ctx *ctx, const float *x, int64_t n, float *y,
                                    void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (n < 0 || (n > 0 && (!x || !y))) return failf(c, SPH_ERR_ARG, "sph_mlp_infer: arguments");
    sph_status rc = ensure_mlp(c);
    if (rc) return rc;
    CK(launch_mlp_infer(c, x, n, y, (cudaStream_t)stream));
    return SPH_OK;
}

extern "C" sph_status sph_bucket_layout(sph_ctx *ctx, int32_t *first, int64_t cap,
                                        int64_t *nslots)
{
    if (!ctx || !nslots) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    *nslots = c.kp.nb;
    if (!first || cap < (int64_t)c.kp.nb + 1)
        return failf(c, SPH_ERR_ARG, "sph_bucket_layout needs %d entries", c.kp.nb + 1);
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(first, c.bstart, sizeof(int) * ((size_t)c.kp.nb + 1), cudaMemcpyDeviceToHost));
    return SPH_OK;
}

extern "C" sph_status sph_set_profiling(sph_ctx *ctx, int32_t on)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    c.prof.on = on != 0;
    c.prof.phase.clear();
    for (int k = 0; k < SPH_PHASE_COUNT; ++k) {
        c.prof.ms[k] = 0.0;
        c.prof.launches[k] = 0;
    }
    return SPH_OK;
}

extern "C" sph_status sph_set_list_arena(sph_ctx *ctx, int64_t entries)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (entries < 0) return failf(c, SPH_ERR_ARG, "arena entries must be >= 0");
    if (c.list_slots + entries > (int64_t)0xffffffffLL)
        return failf(c, SPH_ERR_CAPACITY, "arena of %lld entries exceeds 32-bit list offsets",
                     (long long)entries);
    if (entries > c.arena_alloc) {
        // a larger buffer: lists are rebuilt by every walk, so nothing is
        // copied, but recorded steps point at the old buffer and are dropped
        CK(cudaDeviceSynchronize());
        unsigned *nl = nullptr;
        if (dalloc(&nl, (size_t)(c.list_slots + entries)) != cudaSuccess)
            return failf(c, SPH_ERR_CUDA, "cudaMalloc of the interaction-list arena failed");
        cudaFree(c.list);
        c.list = nl;
        c.arena_alloc = entries;
        for (cudaGraphExec_t *ge : {&c.graph_exec, &c.graph_exec_r})
            if (*ge) cudaGraphExecDestroy(*ge);
        for (cudaGraph_t *gr : {&c.graph, &c.graph_r})
            if (*gr) cudaGraphDestroy(*gr);
        c.graph_exec = c.graph_exec_r = nullptr;
        c.graph = c.graph_r = nullptr;
        c.graph_replayed = false;
        c.density_valid = c.forces_valid = false;
    }
    c.arena_cap = entries;
    return SPH_OK;
}

extern "C" sph_status sph_set_dt_old(sph_ctx *ctx, double dt_old)
{
    if (!ctx) return SPH_ERR_ARG;
    Ctx &c = ctx->c;
    if (!(dt_old >= 0.0) || std::isinf(dt_old)) return failf(c, SPH_ERR_ARG, "dt_old must be >= 0");
    std::vector<double> v(2 * (size_t)c.kp.ninst, dt_old);
    CK(cudaMemcpy(c.dts, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice));
    for (double &d : c.dt_host) d = dt_old;
    c.stats.dt_old = dt_old;
    return SPH_OK;
}

extern "C" sph_status sph_batch_get_dt(const sph_ctx *ctx, double *out)
{
    if (!ctx || !out) return SPH_ERR_ARG;
    std::memcpy(out, ctx->c.dt_host.data(), sizeof(double) * ctx->c.dt_host.size());
    return SPH_OK;
}

extern "C" sph_status sph_get_stats(const sph_ctx *ctx, sph_stats *out)
{
    if (!ctx || !out) return SPH_ERR_ARG;
    *out = ctx->c.stats;
    out->launches = ctx->c.launches;
    for (int k = 0; k < 16; ++k) {
        out->phase_ms[k] = k < SPH_PHASE_COUNT ? ctx->c.prof.ms[k] : 0.0;
        out->phase_launches[k] = k < SPH_PHASE_COUNT ? ctx->c.prof.launches[k] : 0;
    }
    return SPH_OK;
}

extern "C" const char *sph_last_error(const sph_ctx *ctx)
{
    return ctx ? ctx->c.err.c_str() : "NULL context";
}

extern "C" const char *sph_version(void) { return "libsph 0.2 (sm_103a)"; }
