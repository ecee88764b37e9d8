// sph_noalloc.cu -- conserved totals for callers that cannot allocate device memory.
//
// sph_reduce_conserved needs a context, and a context allocates its scratch
// with cudaMalloc.  Some callers cannot do that: an application that hands the
// whole GPU to its own pool allocator and forbids side allocations, a
// monitoring hook called from inside another library's time step (where a
// cudaMalloc would synchronise the device and can fail under memory pressure),
// or code that must not grow the process's device footprint at all.
// sph_reduce_conserved_noalloc gives them the same totals with no allocation:
// the per-block partial sums live in a fixed file-scope device array below.
//
//   * The array holds kNoallocMaxBlocks rows of 9 doubles (576 KiB); every GPU
//     that loads the library keeps it until the process exits.
//   * One block sums kNoallocPerBlock consecutive particles, so n is limited to
//     kNoallocMaxBlocks * kNoallocPerBlock = 8,388,608; larger n is rejected
//     with SPH_ERR_CAPACITY before anything is launched.
//   * Host code cannot use the array's name as a device address.  The address
//     is looked up with cudaGetSymbolAddress in the CUDA context that is
//     current when the call is made (each context that loads the library
//     has its own copy of the array, at its own address) and cached per
//     context.  A call on a stream that is not being captured looks the
//     address up again; a call during a stream capture uses the cached
//     address of its context, so make the first call in each context before
//     any stream capture.
//   * Every call on a device shares the one array and leaves its partials
//     there.  Each call writes every row it later reads, so nothing needs
//     clearing, but calls that overlap on the GPU (different streams, no
//     ordering between them) race on the rows and give wrong totals.
//   * A CUDA error left pending by earlier work of the caller is not consumed:
//     the call returns SPH_ERR_CUDA without launching and leaves the error
//     for the caller to read.
#include <mutex>

#include "sph_internal.cuh"

namespace {

constexpr int kNoallocThreads = 256;
constexpr int kNoallocPerThread = 4;
constexpr int kNoallocPerBlock = kNoallocThreads * kNoallocPerThread;
constexpr int kNoallocMaxBlocks = 8192;
constexpr int kNoallocMaxContexts = 64;

__device__ __align__(256) double g_noalloc_partials[kNoallocMaxBlocks * 9];

// cached device address of the array per CUDA context (context ids are
// unique for the life of the process, so a context created after another was
// destroyed never inherits its entry)
struct ScratchEntry {
    unsigned long long ctx_id;
    double *ptr;
};
std::mutex g_noalloc_mutex;
ScratchEntry g_noalloc_cache[kNoallocMaxContexts] = {};
int g_noalloc_used = 0;

// fixed-order block sums of M, P, L, E_kin, E_int over one slice of particles
__global__ void __launch_bounds__(kNoallocThreads) k_noalloc_partial(
    int n, const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
    const double *__restrict__ vx, const double *__restrict__ vy, const double *__restrict__ vz,
    const double *__restrict__ u, const float *__restrict__ m, double *part)
{
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const int base = blockIdx.x * kNoallocPerBlock;
#pragma unroll
    for (int r = 0; r < kNoallocPerThread; ++r) {
        const int i = base + r * kNoallocThreads + threadIdx.x;
        if (i < n) {
            const double mi = (double)m[i];
            const double p[3] = {x[i], y[i], z[i]}, v[3] = {vx[i], vy[i], vz[i]};
            acc[0] += mi;
            acc[1] += mi * v[0];
            acc[2] += mi * v[1];
            acc[3] += mi * v[2];
            acc[4] += mi * (p[1] * v[2] - p[2] * v[1]);
            acc[5] += mi * (p[2] * v[0] - p[0] * v[2]);
            acc[6] += mi * (p[0] * v[1] - p[1] * v[0]);
            acc[7] += 0.5 * mi * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            acc[8] += mi * u[i];
        }
    }
    __shared__ double sm[9][kNoallocThreads];
#pragma unroll
    for (int k = 0; k < 9; ++k) sm[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int o = kNoallocThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
#pragma unroll
            for (int k = 0; k < 9; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x < 9) part[blockIdx.x * 9 + threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void k_noalloc_final(int nblocks, const double *part, double *out)
{
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (q >= 9) return;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += part[b * 9 + q];
    s = sph::warp_sum(s);
    if (lane == 0) out[q] = s;
}

// id of the CUDA context current on this thread (driver entry points looked
// up once through the runtime, so the library needs no link to libcuda)
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);
bool current_context_id(unsigned long long *id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool resolved = false;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!resolved) {
            cudaDriverEntryPointQueryResult q1, q2;
            void *f1 = nullptr, *f2 = nullptr;
            if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault,
                                                 &q1) == cudaSuccess &&
                q1 == cudaDriverEntryPointSuccess &&
                cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault,
                                                 &q2) == cudaSuccess &&
                q2 == cudaDriverEntryPointSuccess) {
                get_current = (CtxGetCurrentFn)f1;
                get_id = (CtxGetIdFn)f2;
            }
            resolved = true;
        }
    }
    void *ctx = nullptr;
    return get_current && get_id && get_current(&ctx) == 0 && ctx && get_id(ctx, id) == 0;
}

// device address of the partials array in the current context: looked up
// afresh unless the stream is being captured, then from the cache
sph_status noalloc_scratch(cudaStream_t s, double **out)
{
    // (the runtime binds the device's primary context to the thread here if
    // the thread has none yet)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const bool capturing =
        cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone;
    unsigned long long id = 0;
    if (!current_context_id(&id)) return SPH_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    int slot = -1;
    for (int k = 0; k < g_noalloc_used; ++k)
        if (g_noalloc_cache[k].ctx_id == id) slot = k;
    if (capturing) {
        if (slot < 0) return SPH_ERR_CUDA;  // no address known for this context yet
        *out = g_noalloc_cache[slot].ptr;
        return SPH_OK;
    }
    double *ptr = nullptr;
    if (cudaGetSymbolAddress((void **)&ptr, g_noalloc_partials) != cudaSuccess || !ptr)
        return SPH_ERR_CUDA;
    if (slot < 0) {
        // keep the most recent contexts: the oldest entry makes room
        if (g_noalloc_used == kNoallocMaxContexts) {
            for (int k = 1; k < kNoallocMaxContexts; ++k) g_noalloc_cache[k - 1] = g_noalloc_cache[k];
            --g_noalloc_used;
        }
        slot = g_noalloc_used++;
    }
    g_noalloc_cache[slot] = {id, ptr};
    *out = ptr;
    return SPH_OK;
}

}  // namespace

extern "C" sph_status sph_reduce_conserved_noalloc(const sph_particles *p, double *out,
                                                   void *stream)
{
    if (!p || !out || p->n < 0) return SPH_ERR_ARG;
    if (p->n > (int64_t)kNoallocMaxBlocks * kNoallocPerBlock) return SPH_ERR_CAPACITY;
    if (p->n > 0 && (!p->x[0] || !p->x[1] || !p->x[2] || !p->v[0] || !p->v[1] || !p->v[2] ||
                     !p->u || !p->m))
        return SPH_ERR_ARG;
    // an error left by the caller's earlier work is theirs to read: report it
    // without consuming it and launch nothing
    if (cudaPeekAtLastError() != cudaSuccess) return SPH_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    double *part = nullptr;
    sph_status rc = noalloc_scratch(s, &part);
    if (rc != SPH_OK) {
        cudaGetLastError();  // the failed lookup's own error
        return rc;
    }
    const int n = (int)p->n;
    const int nblocks = (n + kNoallocPerBlock - 1) / kNoallocPerBlock;
    if (nblocks > 0)
        k_noalloc_partial<<<nblocks, kNoallocThreads, 0, s>>>(n, p->x[0], p->x[1], p->x[2],
                                                              p->v[0], p->v[1], p->v[2], p->u,
                                                              p->m, part);
    k_noalloc_final<<<1, 288, 0, s>>>(nblocks, part, out);
    // nothing was pending before the launches, so any error now is this call's
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}
