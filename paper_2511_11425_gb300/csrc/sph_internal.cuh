// sph_internal.cuh -- shared declarations of the libsph translation units.
//
// A context holds one or more independent problems ("instances", each with
// its own box, periodicity, gas and viscosity parameters and time step) that
// are stepped together: every phase is ONE launch over all instances.  A
// single problem is a batch of one.
//
// Data layout in device memory (structure of arrays, curve order within each
// instance after sph_build_cells; instances stay in their particle ranges):
//   caller arrays   x,v (f64), u (f64), m,h,rho,omega,a,dudt,... (f32)
//   pinst[i]        instance of particle i (u16)
//   pm[i]           float4 (x - o_b, y - o_b, z - o_b, m): position relative to
//                   the origin o_b of the particle's bucket, plus mass
//   buckets         up to 32 consecutive particles of one instance (one warp)
//                   inside one octree cell of side <= 3 h (slots of an instance
//                   may be empty): first particle bstart[b], instance binst[b], origin
//                   o_b = k_b q with integer grid coordinates k_b (int32 x3) and
//                   the instance's power-of-two quantum q, so origin
//                   differences are exact in f32 and need no FP64
//   tree            per instance an implicit complete binary tree over its
//                   buckets padded to a power of two P (node nbase + k, root
//                   k = 1, leaf of local bucket j = k P + j); each node stores
//                   its cell bound (AABB) and box-of-balls bound as centre /
//                   half-width float4 pairs (Sec. 2.3.2); .w of the cell half
//                   widths = largest bucket extent below, .w of the
//                   box-of-balls half widths = largest h below
//   groups          G <= 8 consecutive bucket slots of one instance (<= 256
//                   particles, inside one cell of side <= 6 h) share one tree
//                   walk: first bucket gfirst[g]
//   lists           per group, kWalkCap slots of source bucket ids
//   pmd[i]          double4_16a, FP64 form only: the same in FP64 (pair sums in FP64)
//   ipos[i]         int4: the same position relative to o_b in fixed point,
//                   units of qx = q 2^-kFixShift (exact integer differences for
//                   the force pairs), .w = h in units of qx (set by the predictor)
//   force records   fpos (rel xyz, h), fvel (v_pred xyz, m), fth (A, c, rho, Omega)
//   accumulators    acc (a xyz, du/dt|Pi), accS (S = sum m_j v_ij.gradW_ij(h_i),
//                   FP64), mumax (max(-mu_ij) as float bits)
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sph.h"

namespace sph {

constexpr int kBucket = 32;       // particles per bucket = one warp
constexpr int kChunk = 128;       // staged candidates processed per chunk
constexpr int kWalkCap = 1024;    // frontier / list entries per group
constexpr int kGroupLog = 3;      // groups of up to 8 buckets
constexpr int kWarpsPerBlock = 4; // pair kernels and walks: 4 warps per block
constexpr int kSortItems = 8;     // keys per thread in a radix-sort tile
constexpr int kSortTile = 256 * kSortItems;  // keys per radix-sort tile
constexpr int kKeyBox = 11;       // doubles per instance of the key box
// Buckets and groups do not straddle large octree cells: consecutive
// particles start a new bucket when their smallest common key cell is wider
// than bucket_cell h, a new group when it is wider than group_cell h
// (defaults below; both are per instance parameters).
constexpr float kKappaBucket = 3.f, kKappaGroup = 6.f;
constexpr int kPadTile = 2048;    // particles per block of the bucket-layout scan

// bucket slots reserved per instance: the plain 32-particle chunks plus half
// as many again for buckets cut short at cell boundaries and group padding
__host__ __device__ inline int64_t bucket_slots(int64_t n)
{
    return n > 0 ? (n + kBucket - 1) / kBucket + (n + 2 * kBucket - 1) / (2 * kBucket) + 8 : 0;
}
constexpr int kMortonBits = 10;   // bits per axis of a curve key (30 bits per instance)
constexpr int kRelistRounds = 3;  // re-walk rounds queued after the first density pass
constexpr int kRoundBlocks = 304; // blocks of a re-walk round's grid-stride launches
constexpr int kBboxChunks = 32;   // blocks per instance for open-axis bounding boxes
constexpr int kConsChunk = 2048;  // particles per block of the conserved totals
// fixed-point positions of the force pairs: qx = q 2^-11, so 2^31 qx = 2^20 q
// is at least half the longest box side (q = 2^(floor(log2 maxext) - 20))
constexpr int kFixShift = 11;
constexpr unsigned kFull = 0xffffffffu;

// learned seed network 4 -> 32 -> 32 -> 1 (parameter offsets in the flat vector)
constexpr int kMlpIn = 4, kMlpHid = 32;
constexpr int kMlpW1 = 0, kMlpB1 = 128, kMlpW2 = 160, kMlpB2 = 1184, kMlpW3 = 1216,
              kMlpB3 = 1248, kMlpParams = 1249;
constexpr int kMlpFragWords = 14 * 32 * 2;  // bf16x2 B fragments of all mma tiles
constexpr float kMlpXScale0 = 100.f, kMlpXScale1 = 4.f, kMlpXScale2 = 100.f,
                kMlpXScale3 = 10.f, kMlpYScale = 100.f;
static_assert(kMlpParams == SPH_MLP_NPARAM, "network size");

enum StatusCode : int {
    ST_OK = 0, ST_ARG = 1, ST_CUDA = 2, ST_CAPACITY = 3, ST_NOCONV = 4, ST_NONFINITE = 5,
    ST_STATE = 7
};

// device-resident status + counters, reset at the start of every API call
struct DevStatus {
    int code;            // first error code raised by a kernel
    int detail;          // what raised it (bucket or particle index, group ...)
    unsigned long long density_pairs;
    unsigned long long force_pairs;
    unsigned long long density_cand;
    unsigned long long force_cand;
    unsigned long long force_av_pairs;
    int max_iters;
    unsigned int relists;                      // groups re-walked in total
    unsigned int redo_cnt[kRelistRounds + 1];  // groups queued for round r
    unsigned int fg_cnt;                       // groups marked by the FastGas pass
};

// one independent problem (device array; every kernel reads its instance)
struct Inst {
    int off, n;          // particles [off, off + n)
    int boff, nb;        // buckets [boff, boff + nb)
    int goff, ng;        // groups [goff, goff + ng)
    int nbase, P, logP;  // tree nodes nbase + [1, 2P)
    int G, logG;         // buckets per group
    int curve;           // SPH_CURVE_*
    float kb, kg;        // bucket / group cell bounds in units of h
    int periodic[3];
    float L[3], invL[3];
    float gamma, alpha, beta, eps_av, eta_courant, eta_acc, n_ngb;
    float eps_abs;       // absolute inflation of f32 bounds (covers rounding)
    float hcap;          // h must stay below half the shortest periodic length
    float qf;            // origin quantum in f32
    float qx, inv_qx;    // fixed-point quantum q 2^-kFixShift and its inverse
    float ic_alpha;      // kernel-imbalance normalisation (interface correction)
    float r_gas[4];      // gas constant per material
    float qx2;           // qx^2
    float fix_lim;       // fixed point usable while bucket extents and h stay below
    unsigned LQ[3];      // periodic length in units of qx (rounded; < 2^32)
    double q, inv_q;     // origin quantum and its inverse (powers of two)
    double lo[3], hi[3], Ld[3], invLd[3];
};

// batch-wide settings (copied by value into every launch)
struct KParams {
    int kernel, energy_mode, max_newton;
    int ninst, n, nb, ng, nnodes;
    int key_passes;      // 8-bit radix passes over (instance, curve index) keys
    int any_open;        // some instance has an open axis
    int fp64;            // SPH_PRECISION_FP64: pair sums and h iteration in FP64
    int evolved;         // SPH_DENSITY_EVOLVED: rho is state (mass conservation)
    int ic;              // interface correction on (Sec. 2.3.4)
    float h_rel_tol, margin;
    float h_step_tol;    // sqrt(h_rel_tol), at most 1e-2: Newton step that ends the iteration
};

// the substep of a hierarchical step that a kernel works on (sph_step_rungs):
// substep `sub` of 2^R of length delta; a particle on rung r has the period
// 2^(R-r) substeps and is active when sub is a multiple of it.  rung = NULL:
// a plain global step.
struct RungArgs {
    const uint8_t *rung;
    int *rmax;
    int sub, R, started;
    double delta, dt0;
};
__host__ __device__ inline bool rung_active(int sub, int R, int r)
{
    return (sub & ((1 << (R - r)) - 1)) == 0;
}

// one block of the bottom-up tree refit: reduce `levels` levels of instance
// `inst` starting at level `lvl`, block index `blk` within that level
struct RefitBlock {
    int inst, lvl, levels, blk;
};

// per-phase device timing of plain calls (sph_set_profiling): an event pair
// around each launch group, read back when the call settles
struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> ev;  // pool: pair k = events 2k, 2k + 1
    std::vector<int> phase;       // phase of each pair recorded in this call
    // the same recorded into the captured steps (event record nodes), per
    // graph: 0 = the re-sorting step, 1 = the refitting step
    std::vector<cudaEvent_t> gev[2];
    std::vector<int> gphase[2];
    int slot = 0;                 // graph being captured
    double ms[SPH_PHASE_COUNT] = {};
    unsigned long long launches[SPH_PHASE_COUNT] = {};
};
constexpr int kProfGraph = 1 << 20;  // prof_begin's index offset for captured pairs

struct Ctx {
    std::vector<sph_params> prm;  // per instance
    std::vector<Inst> inst_host;
    KParams kp;
    int64_t capacity = 0;
    int64_t cap_nb = 0, cap_ng = 0;  // bucket slots and groups the buffers hold
    int device = 0;
    std::string err;
    sph_stats stats{};
    bool cells_valid = false, density_valid = false, forces_valid = false, rho_valid = false;
    int64_t n_built = 0;
    std::vector<double> dt_host;  // per instance step of the last kick-drift-kick

    // instances and their static index maps
    Inst *inst = nullptr;          // device copy of inst_host
    unsigned short *pinst = nullptr;
    int *bstart = nullptr, *binst = nullptr;
    int *gfirst = nullptr;
    int4 *pad_agg = nullptr;       // bucket-layout scan: per tile aggregate / prefix
    int *pad_used = nullptr;       // per instance: bucket slots the layout needs
    RefitBlock *refit = nullptr;   // refit schedule (all bands)
    std::vector<int> refit_band;   // blocks per band (host)

    // status
    DevStatus *st = nullptr;       // device
    DevStatus *st_host = nullptr;  // pinned host mirror
    double *dts = nullptr;         // device per instance [dt_old, dt_new]
    double *dts_host = nullptr;    // pinned mirror
    unsigned int *dtmin = nullptr; // device per instance min_i dt_i as float bits
    double *morton_box = nullptr;  // device per instance key box (kKeyBox doubles)
    double *bbox_part = nullptr;   // device per instance partial min/max for open axes
    double *cons_part = nullptr;   // device per (instance, block) partial sums
    double *cons_out = nullptr;    // device 9 doubles per instance
    double *cons_host = nullptr;   // pinned mirror
    int cons_blocks = 0;           // largest number of blocks of one instance

    // sort
    unsigned long long *keys[2] = {nullptr, nullptr};
    unsigned int *vals[2] = {nullptr, nullptr};
    unsigned int *hist = nullptr;     // 256 x tiles
    unsigned int *digit_tot = nullptr;  // per-digit totals of the current sort pass
    void *tmp = nullptr;              // permutation scratch, 112 B x capacity

    // buckets / tree
    int *origin = nullptr;            // 3 x nb grid coordinates (SoA: kx, ky, kz)
    unsigned int *gflag = nullptr;    // per group: queued for a re-walk
    float4 *node = nullptr;           // 4 float4 per node: box_c, box_r, bob_c, bob_r

    // particle records
    float4 *pm = nullptr;
    double4_16a *pmd = nullptr;   // FP64 form: position relative to the bucket origin, m
    double4_16a *fveld = nullptr; // FP64 form: v_pred xyz, m
    double4_16a *fthd = nullptr;  // FP64 form: A, c, rho, Omega
    double4_16a *acc64 = nullptr; // FP64 form: a xyz, du/dt|Pi
    float4 *fpos = nullptr, *fvel = nullptr, *fth = nullptr;
    int4 *ipos = nullptr;
    float4 *acc = nullptr;
    double *accS = nullptr;
    unsigned *mumax = nullptr;
    float *rho_old = nullptr;
    float *rho_sum = nullptr;         // evolved density mode: the density pass's kernel sum
    float *ic_e = nullptr;            // interface correction: exp(-I^2) per particle
    // hierarchical time steps (sph_step_rungs): rung per particle (permuted
    // with the particles), largest rung of each particle's force partners
    uint8_t *rung = nullptr;
    int *rmax = nullptr;
    // FastGas (Sec. 2.3.6): per bucket "holds an active particle", per group
    // "marked", the queue of marked groups (count in DevStatus::fg_cnt)
    bool fastgas = true;
    uint8_t *bact = nullptr;
    unsigned *gmark = nullptr, *fg_list = nullptr;
    bool rungs_started = false;       // derivatives exist (the first substep has none)
    int rung_R = 0;                   // max_rung of the hierarchical steps so far
    float2 *ic_pt = nullptr;          // interface correction: P, T from the predictor
    bool rho_evolved_init = false;    // p->rho holds an evolved density
    float *h_seed = nullptr;          // density seeds / re-walk seeds

    // lists: kWalkCap slots per group, then an overflow arena of arena_cap
    // entries for groups whose lists outgrow them; list_off[g] = where g's
    // list starts
    unsigned int *list = nullptr, *list_cnt = nullptr, *list_off = nullptr;
    unsigned int *arena_used = nullptr;  // overflow arena entries handed out
    int64_t arena_cap = 0;            // arena entries in use (<= arena_alloc)
    int64_t arena_alloc = 0;          // arena entries allocated behind the slots
    int64_t list_slots = 0;           // fixed list slots (groups x kWalkCap)
    unsigned int *redo = nullptr;     // per round r: group ids queued (ng entries each)

    // host-mode mirror buffers for sph_step_host
    void *mirror = nullptr;
    sph_particles dmirror{};
    // host arrays of the current sph_step_host call and, per array, the
    // address the GPU reaches it at (mapped pinned memory) or NULL (copied by
    // the copy engines instead)
    sph_particles hkey{};
    sph_particles hdev{};

    // learned seed network
    struct Mlp {
        float *w = nullptr;          // FP32 master parameters
        float *m = nullptr, *v = nullptr;  // Adam moments
        uint32_t *frag = nullptr;    // bfloat16 copy as mma B fragments
        float *gpart = nullptr;      // per-block gradient partials (+ loss)
        int64_t gpart_blocks = 0;
        double *loss = nullptr;      // per-step losses of the last training call
        int loss_cap = 0;
        int t = 0;                   // Adam steps taken
        int seed_mode = SPH_SEED_ANALYTIC;
        float dead = 0.f;            // corrections below this (in ln h) are dropped
        bool record = false;
        int stride = 1;
        unsigned step = 0;           // harvest counter (sample selection)
        float *seed0 = nullptr;      // capacity: seeds of the last density pass as given
        float *corr = nullptr;       // capacity: correction of the seed exponent
        float *tfeat = nullptr;      // 4 x capacity inputs of the last kick (SoA)
        float *th = nullptr;         // capacity: h at the last kick (0 = none)
        float *sx = nullptr, *sy = nullptr;  // samples: cap x 4, cap
        unsigned long long *scount = nullptr;  // samples written (device)
        int64_t cap = 0;
    } mlp;

    // captured step
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    sph_particles graph_p{};
    double graph_dt = 0.0;
    uint64_t graph_kernels = 0;   // kernels in one replay
    bool graph_replayed = false;
    bool capturing = false;       // queueing into a stream capture
    cudaGraph_t graph_r = nullptr;          // captured step that only refits
    cudaGraphExec_t graph_exec_r = nullptr;
    uint64_t graph_kernels_r = 0;

    // re-sorting schedule of sph_step and graph replays
    int resort_period = 1;
    int since_sort = 0;           // refit-only steps since the last full build
    bool order_fresh = false;     // a full build ran on this layout
    std::vector<double> graph_totals;  // conserved totals after the last replay

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t kev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    // side stream of the force phase: the predictor runs there beside the
    // force walk (fork and join events; graph edges when captured)
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    // sph_step_host: the step inputs no kernel reads before the end of the
    // density phase are copied in on `copy` while the step starts; the step
    // waits for `late_in` there (an external event-wait node when captured)
    cudaStream_t copy = nullptr;
    cudaEvent_t call0 = nullptr, late_in = nullptr;
    // ... and the outputs final before the step ends are copied back on
    // `copy` once these are reached: density outputs, force outputs; then
    // out_done joins the copy stream back
    cudaEvent_t out_dens = nullptr, out_force = nullptr, out_done = nullptr;
    uint64_t launches = 0;
    Prof prof;
};

// open a timed launch group of `phase` on stream s (returns its pair index,
// offset by kProfGraph while a step is being captured, or -1 when not
// profiling); close it with prof_end
inline int prof_begin(Ctx &c, cudaStream_t s, int phase)
{
    if (!c.prof.on) return -1;
    std::vector<cudaEvent_t> &ev = c.capturing ? c.prof.gev[c.prof.slot] : c.prof.ev;
    std::vector<int> &ph = c.capturing ? c.prof.gphase[c.prof.slot] : c.prof.phase;
    const size_t k = ph.size();
    while (ev.size() < 2 * (k + 1)) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        ev.push_back(e);
    }
    // while capturing, an external record makes an event record node (a
    // plain record would only order the capture's own streams)
    const cudaError_t e = c.capturing ? cudaEventRecordWithFlags(ev[2 * k], s, cudaEventRecordExternal)
                                      : cudaEventRecord(ev[2 * k], s);
    if (e != cudaSuccess) return -1;
    ph.push_back(phase);
    return (int)k + (c.capturing ? kProfGraph : 0);
}
inline void prof_end(Ctx &c, cudaStream_t s, int k)
{
    if (k >= kProfGraph)
        cudaEventRecordWithFlags(c.prof.gev[c.prof.slot][2 * (k - kProfGraph) + 1], s,
                                 cudaEventRecordExternal);
    else if (k >= 0)
        cudaEventRecord(c.prof.ev[2 * k + 1], s);
}

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void raise_status(DevStatus *st, int code, int detail)
{
    if (atomicCAS(&st->code, 0, code) == 0) st->detail = detail;
}

__device__ __forceinline__ float wrapf(float d, float L, float invL)
{
    return d - L * rintf(d * invL);
}

__device__ __forceinline__ double wrapd(double d, double L)
{
    return d - L * rint(d / L);
}

__device__ __forceinline__ void red_add_f64(double *addr, double a)
{
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(addr), "d"(a) : "memory");
}

// vector reduction into global memory (sm_90+): one L2 atomic per 16 bytes
__device__ __forceinline__ void red_add_v4(float4 *addr, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b),
                 "f"(c), "f"(d)
                 : "memory");
}

__device__ __forceinline__ void red_add_f32(float *addr, float a)
{
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(addr), "f"(a) : "memory");
}

template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// overlap of two centre/half-width intervals (on a circle for periodic axes)
__device__ __forceinline__ bool ovl(float ca, float ra, float cb, float rb, bool per, float L,
                                    float invL)
{
    float d = ca - cb;
    if (per) d = wrapf(d, L, invL);
    return fabsf(d) <= ra + rb;
}

// f32 offset o_B - o_A between two bucket origins of one instance (nearest
// periodic image): integer grid difference times the power-of-two quantum,
// exact in f32 whenever the periodic length is a multiple of q
__device__ __forceinline__ float3 origin_offset(const Inst &I, int nb_total,
                                                const int *__restrict__ origin, int A, int B)
{
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float f = (float)(origin[a * nb_total + B] - origin[a * nb_total + A]) * I.qf;
        if (I.periodic[a]) f -= I.L[a] * rintf(f * I.invL[a]);
        d[a] = f;
    }
    return make_float3(d[0], d[1], d[2]);
}

// periodic geometry of one instance, held in registers by the pair kernels
struct PBox {
    int per[3];
    float L[3], invL[3];
};
__device__ __forceinline__ PBox make_pbox(const Inst &I)
{
    PBox b;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        b.per[a] = I.periodic[a];
        b.L[a] = I.L[a];
        b.invL[a] = I.invL[a];
    }
    return b;
}

// bucket -> group (global index) of instance I
__device__ __forceinline__ int group_of(const Inst &I, int b)
{
    return I.goff + ((b - I.boff) >> I.logG);
}

// leaf node (global index) of bucket b of instance I
__device__ __forceinline__ size_t leaf_of(const Inst &I, int b)
{
    return (size_t)I.nbase + I.P + (b - I.boff);
}

// particles in bucket slot b: slots hold consecutive particle ranges, so the
// count is the distance to the next slot's first particle (0 for a padding
// slot; bstart has one sentinel entry past the last slot)
__device__ __forceinline__ int bucket_len(const int *__restrict__ bstart, int b)
{
    const int c = bstart[b + 1] - bstart[b];
    return c < kBucket ? c : kBucket;
}

// Kahan-compensated running sum (the density and force sums accumulate one
// chunk partial at a time; each chunk partial is a short plain f32 sum)
struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// ---------------------------------------------------------------------------
// smoothing kernels, support radius h, dimensionless q = r/h in [0,1):
//   w(q)        kernel shape (normalisation sigma applied by the caller)
//   dwq(q)      w'(q)/q, finite at q = 0 for every kernel here
//   d2w(q)      w''(q) (the first-order move of the h-derivative sum)
// Cubic spline (M4) and Wendland C2/C4/C6 in their 3D forms (Sec. 2.3).
// ---------------------------------------------------------------------------
struct KWC2 {
    static constexpr float sigma = 3.3422538049298023f;  // 21 / (2 pi)
    static constexpr double sigmad = 3.3422538049298023;
    __device__ __forceinline__ static double wd(double q)
    {
        const double t = 1.0 - q, t2 = t * t;
        return t2 * t2 * fma(4.0, q, 1.0);
    }
    __device__ __forceinline__ static double dwqd(double q)
    {
        const double t = 1.0 - q;
        return -20.0 * t * t * t;
    }
    __device__ __forceinline__ static float w(float q)
    {
        float t = 1.f - q, t2 = t * t;
        return t2 * t2 * fmaf(4.f, q, 1.f);
    }
    __device__ __forceinline__ static float dwq(float q)
    {
        float t = 1.f - q;
        return -20.f * t * t * t;
    }
    // the same with 1 - q supplied (t, computed without cancellation)
    __device__ __forceinline__ static float dwqt(float q, float t)
    {
        (void)q;
        return -20.f * t * t * t;
    }
    // w''(q)
    __device__ __forceinline__ static float d2w(float q)
    {
        const float t = 1.f - q;
        return 20.f * t * t * fmaf(4.f, q, -1.f);
    }
    __device__ __forceinline__ static double d2wd(double q)
    {
        const double t = 1.0 - q;
        return 20.0 * t * t * fma(4.0, q, -1.0);
    }
};
struct KWC4 {
    static constexpr float sigma = 4.923856051905513f;  // 495 / (32 pi)
    static constexpr double sigmad = 4.923856051905513;
    __device__ __forceinline__ static double wd(double q)
    {
        const double t = 1.0 - q, t2 = t * t, t6 = t2 * t2 * t2;
        return t6 * fma(q, fma(35.0 / 3.0, q, 6.0), 1.0);
    }
    __device__ __forceinline__ static double dwqd(double q)
    {
        const double t = 1.0 - q, t2 = t * t, t5 = t2 * t2 * t;
        return (-56.0 / 3.0) * t5 * fma(5.0, q, 1.0);
    }
    __device__ __forceinline__ static float w(float q)
    {
        float t = 1.f - q, t2 = t * t, t6 = t2 * t2 * t2;
        return t6 * fmaf(q, fmaf(35.f / 3.f, q, 6.f), 1.f);
    }
    __device__ __forceinline__ static float dwq(float q) { return dwqt(q, 1.f - q); }
    __device__ __forceinline__ static float dwqt(float q, float t)
    {
        float t2 = t * t, t5 = t2 * t2 * t;
        return (-56.f / 3.f) * t5 * fmaf(5.f, q, 1.f);
    }
    __device__ __forceinline__ static float d2w(float q)
    {
        const float t = 1.f - q, t2 = t * t;
        return (-56.f / 3.f) * t2 * t2 * fmaf(q, fmaf(-35.f, q, 4.f), 1.f);
    }
    __device__ __forceinline__ static double d2wd(double q)
    {
        const double t = 1.0 - q, t2 = t * t;
        return (-56.0 / 3.0) * t2 * t2 * fma(q, fma(-35.0, q, 4.0), 1.0);
    }
};
struct KWC6 {
    static constexpr float sigma = 6.788953041263660f;  // 1365 / (64 pi)
    static constexpr double sigmad = 6.788953041263660;
    __device__ __forceinline__ static double wd(double q)
    {
        const double t = 1.0 - q, t2 = t * t, t4 = t2 * t2, t8 = t4 * t4;
        return t8 * fma(q, fma(q, fma(32.0, q, 25.0), 8.0), 1.0);
    }
    __device__ __forceinline__ static double dwqd(double q)
    {
        const double t = 1.0 - q, t2 = t * t, t4 = t2 * t2, t7 = t4 * t2 * t;
        return -22.0 * t7 * fma(q, fma(16.0, q, 7.0), 1.0);
    }
    __device__ __forceinline__ static float w(float q)
    {
        float t = 1.f - q, t2 = t * t, t4 = t2 * t2, t8 = t4 * t4;
        return t8 * fmaf(q, fmaf(q, fmaf(32.f, q, 25.f), 8.f), 1.f);
    }
    __device__ __forceinline__ static float dwq(float q) { return dwqt(q, 1.f - q); }
    __device__ __forceinline__ static float dwqt(float q, float t)
    {
        float t2 = t * t, t4 = t2 * t2, t7 = t4 * t2 * t;
        return -22.f * t7 * fmaf(q, fmaf(16.f, q, 7.f), 1.f);
    }
    __device__ __forceinline__ static float d2w(float q)
    {
        const float t = 1.f - q, t2 = t * t;
        return -22.f * t2 * t2 * t2 * fmaf(q, fmaf(q, fmaf(-160.f, q, -15.f), 6.f), 1.f);
    }
    __device__ __forceinline__ static double d2wd(double q)
    {
        const double t = 1.0 - q, t2 = t * t;
        return -22.0 * t2 * t2 * t2 * fma(q, fma(q, fma(-160.0, q, -15.0), 6.0), 1.0);
    }
};
struct KM4 {
    static constexpr float sigma = 2.5464790894703255f;  // 8 / pi
    static constexpr double sigmad = 2.5464790894703255;
    __device__ __forceinline__ static double wd(double q)
    {
        const double t = 1.0 - q;
        return q < 0.5 ? fma(6.0 * q * q, q - 1.0, 1.0) : 2.0 * t * t * t;
    }
    __device__ __forceinline__ static double dwqd(double q)
    {
        const double t = 1.0 - q;
        return q < 0.5 ? fma(18.0, q, -12.0) : -6.0 * t * t / q;
    }
    __device__ __forceinline__ static float w(float q)
    {
        float t = 1.f - q;
        return q < 0.5f ? fmaf(6.f * q * q, q - 1.f, 1.f) : 2.f * t * t * t;
    }
    __device__ __forceinline__ static float dwq(float q) { return dwqt(q, 1.f - q); }
    __device__ __forceinline__ static float dwqt(float q, float t)
    {
        return q < 0.5f ? fmaf(18.f, q, -12.f) : -6.f * t * t / q;
    }
    __device__ __forceinline__ static float d2w(float q)
    {
        return q < 0.5f ? fmaf(36.f, q, -12.f) : 12.f * (1.f - q);
    }
    __device__ __forceinline__ static double d2wd(double q)
    {
        return q < 0.5 ? fma(36.0, q, -12.0) : 12.0 * (1.0 - q);
    }
};

// dispatch a templated launcher on the runtime kernel id
#define SPH_KERNEL_DISPATCH(kid, KT, ...)           \
    switch (kid) {                                   \
    case SPH_KERNEL_WC2: { using KT = KWC2; __VA_ARGS__; } break; \
    case SPH_KERNEL_WC4: { using KT = KWC4; __VA_ARGS__; } break; \
    case SPH_KERNEL_WC6: { using KT = KWC6; __VA_ARGS__; } break; \
    default: { using KT = KM4; __VA_ARGS__; } break; \
    }

// ---------------------------------------------------------------------------
// host-side launchers (defined in the .cu files); every one queues work on
// stream s and counts its launches in c.launches
// ---------------------------------------------------------------------------
enum WalkMode { WALK_DENSITY = 0, WALK_FORCE = 1 };
// build (sph_build.cu)
cudaError_t launch_build(Ctx &c, const sph_particles &p, cudaStream_t s);
// bounds of the existing buckets refitted to moved particles (no re-sort)
cudaError_t launch_refit(Ctx &c, const sph_particles &p, cudaStream_t s);
cudaError_t launch_bob_refit(Ctx &c, const sph_particles &p, cudaStream_t s);
// group walk: all groups (round < 0) or the groups queued for re-walk round r
cudaError_t launch_walk(Ctx &c, const sph_particles &p, int mode, int round, const float *h_walk,
                        cudaStream_t s);
// the walk of the groups in a device queue (ids, *cnt of them), the overflow
// arena emptied first
cudaError_t launch_walk_queue(Ctx &c, int mode, const unsigned *ids, const unsigned *cnt,
                              const float *h_walk, cudaStream_t s);
// density (sph_density.cu): round < 0 = all buckets, else the buckets of the
// groups queued for round r; fixed_h evaluates at the given h once
cudaError_t launch_density(Ctx &c, const sph_particles &p, const float *h_seed, int round,
                           int fixed_h, int64_t cap, uint32_t *count, int64_t *ids,
                           cudaStream_t s, bool fastgas = false);
cudaError_t launch_isentropic(Ctx &c, const sph_particles &p, cudaStream_t s);
// forces (sph_forces.cu)
cudaError_t launch_predict(Ctx &c, const sph_particles &p, cudaStream_t s,
                           const RungArgs *ra = nullptr);
cudaError_t launch_forces(Ctx &c, const sph_particles &p, cudaStream_t s,
                          const RungArgs *ra = nullptr, bool fastgas = false);
// FastGas (sph_fastgas.cu): mark the groups of the substep's active
// particles and of their neighbours (from the density lists) and queue them
cudaError_t launch_fastgas_mark(Ctx &c, const RungArgs &ra, cudaStream_t s);
cudaError_t launch_forces64(Ctx &c, cudaStream_t s);  // FP64 form (sph_forces64.cu)
// interface correction pass (sph_interface.cu)
cudaError_t launch_interface(Ctx &c, const sph_particles &p, cudaStream_t s);
cudaError_t launch_finalize(Ctx &c, const sph_particles &p, cudaStream_t s,
                            const RungArgs *ra = nullptr);
// integration (sph_integrate.cu)
cudaError_t launch_kdk(Ctx &c, const sph_particles &p, double dt_fixed, cudaStream_t s);
cudaError_t launch_conserved(Ctx &c, const sph_particles &p, cudaStream_t s);
// hierarchical step: kicks of the active particles, rung choice, drift of all
cudaError_t launch_kdk_rungs(Ctx &c, const sph_particles &p, const RungArgs &ra, cudaStream_t s);
// permute the rungs with the particles at a full build
cudaError_t launch_rung_permute(Ctx &c, const unsigned *perm, int n, cudaStream_t s);
// learned seed (sph_mlp.cu)
cudaError_t launch_mlp_permute(Ctx &c, const unsigned *perm, int n, cudaStream_t s);
cudaError_t launch_mlp_harvest(Ctx &c, const sph_particles &p, cudaStream_t s);
cudaError_t launch_mlp_seed(Ctx &c, const sph_particles &p, cudaStream_t s);
cudaError_t launch_mlp_pack(Ctx &c, cudaStream_t s);
int mlp_grad_blocks(long long batch);
cudaError_t launch_mlp_grad(Ctx &c, const float *sx, const float *sy, long long count,
                            long long batch, int random, unsigned long long seed, int iter,
                            cudaStream_t s);
cudaError_t launch_mlp_update(Ctx &c, long long batch, int adam, double lr, float *grad_out,
                              double *loss, cudaStream_t s);
cudaError_t launch_mlp_infer(Ctx &c, const float *x, long long n, float *y, cudaStream_t s);

// ---------------------------------------------------------------------------
// warp-level inference of the seed network on the tensor cores: lane p of
// the warp supplies the 4 inputs of its particle (zeros when it has none)
// and receives the network output.  The 32 particles form two 16-row tiles;
// each layer is a chain of mma.m16n8k16 (bfloat16 operands, FP32
// accumulation) whose accumulator fragments are, after bias and ReLU,
// exactly the A fragments of the next layer, so activations never leave
// the registers.  frag holds the weights as B fragments: tile t, lane l,
// word r at frag[(t * 32 + l) * 2 + r]; tiles 0-3 = layer 1 (n-tile j),
// 4-11 = layer 2 (n-tile j, k-tile kk at 4 + 2 j + kk), 12-13 = layer 3.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&b);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1,
                                               uint32_t a2, uint32_t a3, uint32_t b0,
                                               uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
        "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float mlp_warp_infer(const uint32_t *__restrict__ frag,
                                                const float *__restrict__ w, float x0, float x1,
                                                float x2, float x3, int lane)
{
    const int g = lane >> 2, t = lane & 3;
    const uint32_t p01 = pack_bf16x2(x0, x1), p23 = pack_bf16x2(x2, x3);
    float out[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        // layer 1: A = inputs (k = 0..3, zero beyond), one k-tile
        const uint32_t lo01 = __shfl_sync(kFull, p01, 16 * mt + g);
        const uint32_t lo23 = __shfl_sync(kFull, p23, 16 * mt + g);
        const uint32_t hi01 = __shfl_sync(kFull, p01, 16 * mt + g + 8);
        const uint32_t hi23 = __shfl_sync(kFull, p23, 16 * mt + g + 8);
        const uint32_t a0 = t == 0 ? lo01 : (t == 1 ? lo23 : 0u);
        const uint32_t a1 = t == 0 ? hi01 : (t == 1 ? hi23 : 0u);
        uint32_t A[2][4];  // A fragments of the next layer, per k-tile
        {
            float d[4][4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint2 b = *reinterpret_cast<const uint2 *>(frag + (j * 32 + lane) * 2);
                const float bb0 = w[kMlpB1 + 8 * j + 2 * t], bb1 = w[kMlpB1 + 8 * j + 2 * t + 1];
                d[j][0] = bb0; d[j][1] = bb1; d[j][2] = bb0; d[j][3] = bb1;
                mma_bf16_16816(d[j], a0, a1, 0u, 0u, b.x, b.y);
            }
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                A[kk][0] = pack_bf16x2(fmaxf(d[2 * kk][0], 0.f), fmaxf(d[2 * kk][1], 0.f));
                A[kk][1] = pack_bf16x2(fmaxf(d[2 * kk][2], 0.f), fmaxf(d[2 * kk][3], 0.f));
                A[kk][2] = pack_bf16x2(fmaxf(d[2 * kk + 1][0], 0.f), fmaxf(d[2 * kk + 1][1], 0.f));
                A[kk][3] = pack_bf16x2(fmaxf(d[2 * kk + 1][2], 0.f), fmaxf(d[2 * kk + 1][3], 0.f));
            }
        }
        // layer 2: 4 n-tiles x 2 k-tiles
        {
            float d[4][4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float bb0 = w[kMlpB2 + 8 * j + 2 * t], bb1 = w[kMlpB2 + 8 * j + 2 * t + 1];
                d[j][0] = bb0; d[j][1] = bb1; d[j][2] = bb0; d[j][3] = bb1;
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    const uint2 b =
                        *reinterpret_cast<const uint2 *>(frag + ((4 + 2 * j + kk) * 32 + lane) * 2);
                    mma_bf16_16816(d[j], A[kk][0], A[kk][1], A[kk][2], A[kk][3], b.x, b.y);
                }
            }
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                A[kk][0] = pack_bf16x2(fmaxf(d[2 * kk][0], 0.f), fmaxf(d[2 * kk][1], 0.f));
                A[kk][1] = pack_bf16x2(fmaxf(d[2 * kk][2], 0.f), fmaxf(d[2 * kk][3], 0.f));
                A[kk][2] = pack_bf16x2(fmaxf(d[2 * kk + 1][0], 0.f), fmaxf(d[2 * kk + 1][1], 0.f));
                A[kk][3] = pack_bf16x2(fmaxf(d[2 * kk + 1][2], 0.f), fmaxf(d[2 * kk + 1][3], 0.f));
            }
        }
        // layer 3: one n-tile whose column 0 is the output
        {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const uint2 b = *reinterpret_cast<const uint2 *>(frag + ((12 + kk) * 32 + lane) * 2);
                mma_bf16_16816(d, A[kk][0], A[kk][1], A[kk][2], A[kk][3], b.x, b.y);
            }
            out[mt][0] = d[0];  // row g, column 2t (column 0 on lanes with t == 0)
            out[mt][1] = d[2];  // row g + 8
        }
    }
    // row r of tile mt sits on lane 4 (r mod 8), register (r >= 8)
    const int mt = lane >> 4, r = lane & 15, src = 4 * (r & 7);
    const float v00 = __shfl_sync(kFull, out[0][0], src), v01 = __shfl_sync(kFull, out[0][1], src);
    const float v10 = __shfl_sync(kFull, out[1][0], src), v11 = __shfl_sync(kFull, out[1][1], src);
    const float y = mt == 0 ? (r < 8 ? v00 : v01) : (r < 8 ? v10 : v11);
    return y + w[kMlpB3];
}

}  // namespace sph
