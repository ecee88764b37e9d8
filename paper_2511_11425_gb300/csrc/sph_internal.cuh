// sph_internal.cuh -- shared declarations of the libsph translation units.
//
// Data layout in device memory (structure of arrays, Morton order after
// sph_build_cells):
//   caller arrays   x,v (f64), u (f64), m,h,rho,omega,a,dudt,... (f32)
//   pm[i]           float4 (x - o_b, y - o_b, z - o_b, m): position relative to
//                   the origin o_b of the particle's bucket, plus mass
//   buckets         32 consecutive particles; origin o_b = k_b q with integer
//                   grid coordinates k_b (int32 x3) and the power-of-two quantum
//                   q, so origin differences are exact in f32 and need no FP64
//   groups          G = 8 consecutive buckets (256 particles) share one walk
//   tree            implicit complete binary tree over the buckets padded to a
//                   power of two P (root 1, leaf of bucket b = P + b); each node
//                   stores its cell bound (AABB) and box-of-balls bound as
//                   centre/half-width float4 pairs, Sec. 2.3.2
//   lists           per group, the source buckets whose bounds overlap the
//                   group's bounds (CSR: start/count per group into one u32
//                   array); each sink bucket filters them against its own bounds
//   force records   fpos (rel xyz, h), fvel (v_pred xyz, m), fth (A, c, rho, -)
//   accumulators    acc (a xyz, S = sum m_j v_ij.gradW_ij(h_i)), acc2 (du/dt|Pi,
//                   max(-mu_ij) as float bits)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/sph.h"

namespace sph {

constexpr int kBucket = 32;       // particles per bucket = one warp
constexpr int kChunk = 128;       // staged candidates processed per chunk
constexpr int kWalkCap = 1024;    // frontier / list entries per sink bucket
constexpr int kWarpsPerBlock = 4; // pair kernels and walks: 4 warps per block
constexpr int kSortItems = 8;     // keys per thread in a radix-sort tile
constexpr int kSortTile = 256 * kSortItems;  // keys per radix-sort tile
constexpr int kMortonBits = 10;   // bits per axis of the Morton key (30-bit keys)
constexpr int kSortPasses = 4;    // 8-bit digits cover the 30-bit keys
constexpr unsigned kFull = 0xffffffffu;

enum StatusCode : int {
    ST_OK = 0, ST_ARG = 1, ST_CUDA = 2, ST_CAPACITY = 3, ST_NOCONV = 4, ST_NONFINITE = 5,
    ST_TIMEOUT = 6, ST_STATE = 7
};

// device-resident status + counters, reset at the start of every API call
struct DevStatus {
    int code;            // first error code raised by a kernel
    int detail;          // what raised it (bucket or particle index, needed size ...)
    unsigned long long density_pairs;
    unsigned long long force_pairs;
    unsigned long long density_cand;
    unsigned long long force_cand;
    unsigned long long force_av_pairs;
    int max_iters;
    unsigned int redo_count;   // buckets whose h left the list coverage
    unsigned int list_used;    // entries allocated in the list buffer
    unsigned int list_need;    // entries the walk wanted (>= list_used on overflow)
    unsigned int dt_min_bits;  // min_i dt_i as float bits (positive floats order as ints)
    unsigned int pad;
};

// parameters as the kernels see them (copied by value into every launch)
struct KParams {
    int kernel, energy_mode, max_newton, nb, P, logP;
    int G, logG, ng;      // buckets per group, log2, number of groups
    int periodic[3];
    int n;
    float L[3], invL[3], halfL[3];
    float n_ngb, gamma, alpha, beta, eps_av, eta_courant, eta_acc, h_rel_tol, margin;
    float eps_abs;        // absolute inflation of f32 bounds (covers rounding)
    float hcap;           // h must stay below half the shortest periodic length
    double q, inv_q;      // origin quantum and its inverse (powers of two)
    float qf;             // q in f32
    double Ld[3], invLd[3];  // periodic lengths in FP64
    double lo[3], hi[3];  // box
};

struct Ctx {
    sph_params prm;
    KParams kp;
    int64_t capacity = 0;
    int device = 0;
    std::string err;
    sph_stats stats{};
    bool cells_valid = false, density_valid = false, forces_valid = false, rho_valid = false;
    int64_t n_built = 0;

    // status
    DevStatus *st = nullptr;       // device
    DevStatus *st_host = nullptr;  // pinned host mirror
    double *dts = nullptr;         // device [dt_old, dt_new]
    unsigned int *dtmin = nullptr; // device min_i dt_i as float bits
    double *morton_box = nullptr;  // device [lo0,lo1,lo2, inv0,inv1,inv2]
    double *bbox_part = nullptr;   // device partial min/max for open axes
    double *cons_part = nullptr;   // device partial sums for sph_reduce_conserved
    double *cons_out = nullptr;    // device 9 doubles

    // sort
    unsigned int *keys[2] = {nullptr, nullptr};
    unsigned int *vals[2] = {nullptr, nullptr};
    unsigned int *hist = nullptr;     // 256 x tiles
    unsigned int *digit_tot = nullptr;  // per-digit totals of the current sort pass
    void *tmp = nullptr;              // permutation scratch, 112 B x capacity
    unsigned int *perm = nullptr;     // final permutation (sorted -> old index)

    // buckets / tree
    int nb_cap = 0, P_cap = 0;
    int *origin = nullptr;            // 3 x nb grid coordinates (SoA: kx, ky, kz)
    unsigned int *gflag = nullptr;    // per group: queued for a re-walk
    float4 *node = nullptr;           // 4 float4 per node: box_c, box_r, bob_c, bob_r

    // particle records
    float4 *pm = nullptr;
    float4 *fpos = nullptr, *fvel = nullptr, *fth = nullptr;
    float4 *acc = nullptr;
    float2 *acc2 = nullptr;
    float *rho_old = nullptr;
    float *h_seed = nullptr;          // density seeds / redo seeds

    // lists
    unsigned int *list_start = nullptr, *list_cnt = nullptr, *list = nullptr;
    int64_t list_cap = 0;
    unsigned int *redo = nullptr;     // ids of groups queued for a re-walk (2 halves)

    // host-mode mirror buffers for sph_step_host
    void *mirror = nullptr;
    sph_particles dmirror{};

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t kev[3] = {nullptr, nullptr, nullptr};  // walk start / kernel start / kernel end
    uint64_t launches = 0;
};

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

// f32 offset o_B - o_A between two bucket origins (nearest periodic image):
// integer grid difference times the power-of-two quantum, exact in f32
__device__ __forceinline__ float3 origin_offset(const KParams &kp, const int *__restrict__ origin,
                                                int A, int B)
{
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float f = (float)(origin[a * kp.nb + B] - origin[a * kp.nb + A]) * kp.qf;
        if (kp.periodic[a]) f -= kp.L[a] * rintf(f * kp.invL[a]);
        d[a] = f;
    }
    return make_float3(d[0], d[1], d[2]);
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
// Cubic spline (M4) and Wendland C2/C4/C6 in their 3D forms (Sec. 2.3).
// ---------------------------------------------------------------------------
struct KWC2 {
    static constexpr float sigma = 3.3422538049298023f;  // 21 / (2 pi)
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
};
struct KWC4 {
    static constexpr float sigma = 4.923856051905513f;  // 495 / (32 pi)
    __device__ __forceinline__ static float w(float q)
    {
        float t = 1.f - q, t2 = t * t, t6 = t2 * t2 * t2;
        return t6 * fmaf(q, fmaf(35.f / 3.f, q, 6.f), 1.f);
    }
    __device__ __forceinline__ static float dwq(float q)
    {
        float t = 1.f - q, t2 = t * t, t5 = t2 * t2 * t;
        return (-56.f / 3.f) * t5 * fmaf(5.f, q, 1.f);
    }
};
struct KWC6 {
    static constexpr float sigma = 6.788953041263660f;  // 1365 / (64 pi)
    __device__ __forceinline__ static float w(float q)
    {
        float t = 1.f - q, t2 = t * t, t4 = t2 * t2, t8 = t4 * t4;
        return t8 * fmaf(q, fmaf(q, fmaf(32.f, q, 25.f), 8.f), 1.f);
    }
    __device__ __forceinline__ static float dwq(float q)
    {
        float t = 1.f - q, t2 = t * t, t4 = t2 * t2, t7 = t4 * t2 * t;
        return -22.f * t7 * fmaf(q, fmaf(16.f, q, 7.f), 1.f);
    }
};
struct KM4 {
    static constexpr float sigma = 2.5464790894703255f;  // 8 / pi
    __device__ __forceinline__ static float w(float q)
    {
        float t = 1.f - q;
        return q < 0.5f ? fmaf(6.f * q * q, q - 1.f, 1.f) : 2.f * t * t * t;
    }
    __device__ __forceinline__ static float dwq(float q)
    {
        float t = 1.f - q;
        return q < 0.5f ? fmaf(18.f, q, -12.f) : -6.f * t * t / q;
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
// host-side launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
// build (sph_build.cu)
cudaError_t launch_build(Ctx &c, const sph_particles &p, cudaStream_t s);
cudaError_t launch_bob_refit(Ctx &c, const sph_particles &p, cudaStream_t s);
cudaError_t launch_walk(Ctx &c, const sph_particles &p, int mode, const unsigned int *group_ids,
                        int ngroups, const float *h_for_walk, cudaStream_t s);
// density (sph_density.cu)
cudaError_t launch_density(Ctx &c, const sph_particles &p, const float *h_seed,
                           const unsigned int *bucket_ids, int nbuckets, int fixed_h,
                           int64_t cap, uint32_t *count, int64_t *ids, cudaStream_t s);
cudaError_t launch_isentropic(Ctx &c, const sph_particles &p, cudaStream_t s);
// forces (sph_forces.cu)
cudaError_t launch_predict(Ctx &c, const sph_particles &p, cudaStream_t s);
cudaError_t launch_forces(Ctx &c, const sph_particles &p, cudaStream_t s);
cudaError_t launch_finalize(Ctx &c, const sph_particles &p, cudaStream_t s);
// integration (sph_integrate.cu)
cudaError_t launch_kdk(Ctx &c, const sph_particles &p, double dt_fixed, cudaStream_t s);
cudaError_t launch_conserved(Ctx &c, const sph_particles &p, cudaStream_t s);

enum WalkMode { WALK_DENSITY = 0, WALK_FORCE = 1 };

}  // namespace sph
