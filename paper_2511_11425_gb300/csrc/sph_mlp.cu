// sph_mlp.cu -- the learned seed of the smoothing-length iteration.
//
// The paper runs Newton-Raphson on the constant kernel mass for every h
// (Sec. 2.3.3) and does not say where it starts.  Here a 4-32-32-1 ReLU
// network proposes the start (the correction to the continuity estimate
// h exp(dt divv / 3)); inference runs inside the kick-drift-kick
// (mlp_warp_infer: bfloat16 tensor-core mma, FP32 accumulation), training
// runs here: FP32 forward and backward over minibatches of samples that the
// simulation records from its own converged h, gradients summed in a fixed
// order, Adam updates of the FP32 master copy, and a repack of the bfloat16
// inference copy.  The paper has no counterpart for the network.
#include "sph_internal.cuh"

namespace sph {

constexpr int kMlpBlock = 128;               // samples per chunk (one per thread)
constexpr int kMlpPart = kMlpParams + 1;     // gradient partial + loss partial
constexpr int kMlpPerThread = (kMlpPart + kMlpBlock - 1) / kMlpBlock;  // 10
constexpr int kMlpMaxBlocks = 1024;
constexpr int kMlpRow = 33;                  // padded row of the shared activations

// shared memory of the training kernel (dynamic, opt-in above 48 KB)
struct MlpShared {
    float w[kMlpParams + 3];
    float x[kMlpBlock][4];
    float a1[kMlpBlock][kMlpRow];   // relu(z1)
    float d1[kMlpBlock][kMlpRow];   // dL/dz1
    float a2[kMlpBlock][kMlpRow];   // relu(z2)
    float d2[kMlpBlock][kMlpRow];   // dL/dz2
    float dout[kMlpBlock];          // dL/dout
    float r2[kMlpBlock];            // squared residual
};

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// MurmurHash3's 32-bit finaliser: sample selection of the harvest
__device__ __forceinline__ unsigned fmix32(unsigned h)
{
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// bfloat16 B fragments of every mma tile (layout in sph_internal.cuh)
__global__ void k_mlp_pack(const float *__restrict__ w, uint32_t *frag)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= kMlpFragWords) return;
    const int tile = idx >> 6, lane = (idx >> 1) & 31, r = idx & 1;
    const int g = lane >> 2, t = lane & 3;
    float lo = 0.f, hi = 0.f;
    if (tile < 4) {  // layer 1: B[k][n] = W1[n][k], k < 4 only
        const int n = 8 * tile + g, k = 2 * t;
        if (r == 0 && k < kMlpIn) {
            lo = w[kMlpW1 + n * kMlpIn + k];
            hi = w[kMlpW1 + n * kMlpIn + k + 1];
        }
    } else if (tile < 12) {  // layer 2: B[k][n] = W2[n][k]
        const int q = tile - 4, j = q >> 1, kk = q & 1;
        const int n = 8 * j + g, k = 16 * kk + 2 * t + 8 * r;
        lo = w[kMlpW2 + n * kMlpHid + k];
        hi = w[kMlpW2 + n * kMlpHid + k + 1];
    } else {  // layer 3: B[k][0] = W3[k], other columns zero
        const int kk = tile - 12, k = 16 * kk + 2 * t + 8 * r;
        if (g == 0) {
            lo = w[kMlpW3 + k];
            hi = w[kMlpW3 + k + 1];
        }
    }
    frag[idx] = pack_bf16x2(lo, hi);
}

// the records written by the last kick move with the particles
__global__ void k_mlp_gather(const unsigned *__restrict__ perm, int n, int cap,
                             const float *__restrict__ tfeat, const float *__restrict__ th,
                             float *tmp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned j = perm[i];
#pragma unroll
    for (int a = 0; a < 4; ++a) tmp[(size_t)a * n + i] = tfeat[(size_t)a * cap + j];
    tmp[(size_t)4 * n + i] = th[j];
}

__global__ void k_mlp_scatter_back(int n, int cap, const float *__restrict__ tmp, float *tfeat,
                                   float *th)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int a = 0; a < 4; ++a) tfeat[(size_t)a * cap + i] = tmp[(size_t)a * n + i];
    th[i] = tmp[(size_t)4 * n + i];
}

// after the density pass: records + converged h -> training samples
__global__ void k_mlp_harvest(int n, int cap, const float *__restrict__ tfeat,
                              const float *__restrict__ th, const float *__restrict__ h,
                              unsigned step, unsigned stride, long long scap, float *sx,
                              float *sy, unsigned long long *scount)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float h0 = th[i];
    if (!(h0 > 0.f)) return;
    if (fmix32((unsigned)i * 0x9E3779B9u ^ step * 0x85EBCA6Bu) % stride != 0u) return;
    const float lr = logf(h[i] / h0);
    if (!(fabsf(lr) <= 0.6931472f)) return;
    float x[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) x[a] = tfeat[(size_t)a * cap + i];
    const float y = kMlpYScale * (lr - x[0] * (1.f / kMlpXScale0));
    const unsigned long long slot = atomicAdd(scount, 1ull) % (unsigned long long)scap;
#pragma unroll
    for (int a = 0; a < 4; ++a) sx[slot * 4 + a] = x[a];
    sy[slot] = y;
}

// FP32 forward + backward of chunks of 128 samples; block b takes chunks
// b, b + gridDim.x, ... and writes its summed gradient (and squared-residual
// sum) to part[b].  The sample of batch slot j is j itself (full batch) or
// floor(count * u / 2^64) with u = SplitMix64(seed + (iter << 32) + j).
__global__ void __launch_bounds__(kMlpBlock) k_mlp_grad(
    const float *__restrict__ w, const float *__restrict__ sx, const float *__restrict__ sy,
    long long count, long long batch, int random, unsigned long long seed, int iter, float *part)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpShared &S = *reinterpret_cast<MlpShared *>(smem_raw);
    const int tid = threadIdx.x;
    for (int p = tid; p < kMlpParams; p += kMlpBlock) S.w[p] = w[p];
    float acc[kMlpPerThread];
#pragma unroll
    for (int m = 0; m < kMlpPerThread; ++m) acc[m] = 0.f;
    const float inv_b = 2.f / (float)batch;
    const long long nchunks = (batch + kMlpBlock - 1) / kMlpBlock;
    __syncthreads();
    for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const long long j = ch * kMlpBlock + tid;
        const bool valid = j < batch;
        float x[4] = {0.f, 0.f, 0.f, 0.f}, yv = 0.f;
        if (valid) {
            long long s = j;
            if (random) {
                const unsigned long long u =
                    splitmix64(seed + ((unsigned long long)(unsigned)iter << 32) +
                               (unsigned long long)j);
                s = (long long)__umul64hi(u, (unsigned long long)count);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) x[a] = sx[s * 4 + a];
            yv = sy[s];
        }
        // forward: a1 in registers and shared memory, a2 in shared memory
        float a1[kMlpHid];
#pragma unroll
        for (int q = 0; q < kMlpHid; ++q) {
            float t = S.w[kMlpB1 + q];
#pragma unroll
            for (int a = 0; a < 4; ++a) t = fmaf(S.w[kMlpW1 + q * 4 + a], x[a], t);
            a1[q] = fmaxf(t, 0.f);
            S.a1[tid][q] = a1[q];
        }
        float out = S.w[kMlpB3];
#pragma unroll 4
        for (int q = 0; q < kMlpHid; ++q) {
            float t = S.w[kMlpB2 + q];
#pragma unroll
            for (int k = 0; k < kMlpHid; ++k) t = fmaf(S.w[kMlpW2 + q * kMlpHid + k], a1[k], t);
            const float a = fmaxf(t, 0.f);
            S.a2[tid][q] = a;
            out = fmaf(S.w[kMlpW3 + q], a, out);
        }
        const float r = valid ? out - yv : 0.f;
        const float dout = inv_b * r;
        // backward: dL/dz2 (ReLU mask from a2 > 0), then dL/dz1
        float d1[kMlpHid];
#pragma unroll
        for (int k = 0; k < kMlpHid; ++k) d1[k] = 0.f;
#pragma unroll 4
        for (int q = 0; q < kMlpHid; ++q) {
            const float d2 = S.a2[tid][q] > 0.f ? dout * S.w[kMlpW3 + q] : 0.f;
            S.d2[tid][q] = d2;
#pragma unroll
            for (int k = 0; k < kMlpHid; ++k) d1[k] = fmaf(d2, S.w[kMlpW2 + q * kMlpHid + k], d1[k]);
        }
#pragma unroll
        for (int k = 0; k < kMlpHid; ++k) S.d1[tid][k] = a1[k] > 0.f ? d1[k] : 0.f;
#pragma unroll
        for (int a = 0; a < 4; ++a) S.x[tid][a] = x[a];
        S.dout[tid] = dout;
        S.r2[tid] = r * r;
        __syncthreads();
        // parameter p sums its terms over the chunk's samples in order
#pragma unroll
        for (int m = 0; m < kMlpPerThread; ++m) {
            const int p = tid + m * kMlpBlock;
            if (p >= kMlpPart) break;
            float t = 0.f;
            if (p < kMlpB1) {
                const int q = p >> 2, a = p & 3;
                for (int s = 0; s < kMlpBlock; ++s) t = fmaf(S.d1[s][q], S.x[s][a], t);
            } else if (p < kMlpW2) {
                const int q = p - kMlpB1;
                for (int s = 0; s < kMlpBlock; ++s) t += S.d1[s][q];
            } else if (p < kMlpB2) {
                const int q = (p - kMlpW2) >> 5, k = (p - kMlpW2) & 31;
                for (int s = 0; s < kMlpBlock; ++s) t = fmaf(S.d2[s][q], S.a1[s][k], t);
            } else if (p < kMlpW3) {
                const int q = p - kMlpB2;
                for (int s = 0; s < kMlpBlock; ++s) t += S.d2[s][q];
            } else if (p < kMlpB3) {
                const int k = p - kMlpW3;
                for (int s = 0; s < kMlpBlock; ++s) t = fmaf(S.dout[s], S.a2[s][k], t);
            } else if (p == kMlpB3) {
                for (int s = 0; s < kMlpBlock; ++s) t += S.dout[s];
            } else {
                for (int s = 0; s < kMlpBlock; ++s) t += S.r2[s];
            }
            acc[m] += t;
        }
        __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < kMlpPerThread; ++m) {
        const int p = tid + m * kMlpBlock;
        if (p < kMlpPart) part[(size_t)blockIdx.x * kMlpPart + p] = acc[m];
    }
}

// fold the block partials (in block order, FP64) and either take an Adam
// step or write the gradient; the loss of the step goes to *loss
__global__ void k_mlp_update(const float *__restrict__ part, int nblocks, long long batch,
                             int adam, float *w, float *m, float *v, double lr_t, double beta1,
                             double beta2, double eps_t, float *grad_out, double *loss)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kMlpPart) return;
    double g = 0.0;
    for (int b = 0; b < nblocks; ++b) g += (double)part[(size_t)b * kMlpPart + p];
    if (p == kMlpParams) {
        *loss = g / (double)batch;
        return;
    }
    if (!adam) {
        grad_out[p] = (float)g;
        return;
    }
    // Adam with the bias corrections folded into lr_t and eps_t
    const double mn = beta1 * (double)m[p] + (1.0 - beta1) * g;
    const double vn = beta2 * (double)v[p] + (1.0 - beta2) * g * g;
    m[p] = (float)mn;
    v[p] = (float)vn;
    w[p] = (float)((double)w[p] - lr_t * mn / (sqrt(vn) + eps_t));
}

// network outputs for rows of inputs (the tensor-core path of the seed)
__global__ void __launch_bounds__(128) k_mlp_infer(const uint32_t *__restrict__ frag,
                                                   const float *__restrict__ w,
                                                   const float *__restrict__ x, long long n,
                                                   float *y)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    float f[4] = {0.f, 0.f, 0.f, 0.f};
    if (valid) {
#pragma unroll
        for (int a = 0; a < 4; ++a) f[a] = x[i * 4 + a];
    }
    const float out = mlp_warp_infer(frag, w, f[0], f[1], f[2], f[3], threadIdx.x & 31);
    if (valid) y[i] = out;
}

// Network inputs of every particle at the end of a step (after the step size
// is chosen, before the kick moves h): MODE bit 1 records them with h for the
// next harvest, bit 0 runs the network and leaves the correction of the
// continuity exponent in corr[i] (0 where it is not applied: a particle at
// rest within the Newton tolerance, a correction inside the dead zone, a
// non-finite output).  Warps whose particles are all at rest skip the
// network.
template <int MODE>
__global__ void __launch_bounds__(128) k_mlp_seed(
    KParams kp, int n, const Inst *__restrict__ insts, const unsigned short *__restrict__ pinst,
    const float *__restrict__ h, const float *__restrict__ divv,
    const unsigned short *__restrict__ nngb, const float *__restrict__ seed0,
    const double *__restrict__ dts, const uint32_t *__restrict__ frag,
    const float *__restrict__ w, float dead, int cap, float *tfeat, float *th, float *corr,
    const DevStatus *st)
{
    if (st->code != 0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = i < n;
    float xin[4] = {0.f, 0.f, 0.f, 0.f};
    if (valid) {
        const int k = pinst[i];
        const double dt_old = dts[2 * k], dt_new = dts[2 * k + 1];
        const float hi = h[i];
        xin[0] = kMlpXScale0 * ((float)dt_new * divv[i] * (1.f / 3.f));
        xin[1] = kMlpXScale1 * ((float)nngb[i] / insts[k].n_ngb - 1.f);
        const float sd = seed0[i];
        xin[2] = sd > 0.f ? kMlpXScale2 * logf(hi / sd) : 0.f;
        // FP32 on purpose: a per-particle FP64 log costs more than the network
        xin[3] = dt_old > 0.0 ? kMlpXScale3 * logf((float)dt_new / (float)dt_old) : 0.f;
        if (MODE & 2) {
#pragma unroll
            for (int a = 0; a < 4; ++a) tfeat[(size_t)a * cap + i] = xin[a];
            th[i] = hi;
        }
    }
    if (!(MODE & 1)) return;
    const float rest = kMlpXScale0 * kp.h_rel_tol;
    const bool at_rest = !valid || (fabsf(xin[0]) < rest && fabsf(xin[2]) < rest);
    float y = 0.f;
    if (!__all_sync(kFull, at_rest)) {  // warp-uniform
        y = mlp_warp_infer(frag, w, xin[0], xin[1], xin[2], xin[3], lane) * (1.f / kMlpYScale);
        if (!isfinite(y) || at_rest || fabsf(y) < dead) y = 0.f;
    }
    if (valid) corr[i] = y;
}

// ---- launchers ---------------------------------------------------------------
cudaError_t launch_mlp_seed(Ctx &c, const sph_particles &p, cudaStream_t s)
{
    const int n = (int)p.n;
    const int mode = (c.mlp.seed_mode == SPH_SEED_MLP ? 1 : 0) | (c.mlp.record ? 2 : 0);
    if (mode == 0 || n == 0) return cudaSuccess;
    const int g = (n + 127) / 128;
    c.launches += 1;
#define SPH_SEED(M)                                                                           \
    k_mlp_seed<M><<<g, 128, 0, s>>>(c.kp, n, c.inst, c.pinst, p.h, p.divv, p.nngb, c.mlp.seed0, \
                                    c.dts, c.mlp.frag, c.mlp.w, c.mlp.dead, (int)c.capacity, \
                                    c.mlp.tfeat, c.mlp.th, c.mlp.corr, c.st)
    if (mode == 1) SPH_SEED(1);
    else if (mode == 2) SPH_SEED(2);
    else SPH_SEED(3);
#undef SPH_SEED
    return cudaGetLastError();
}

cudaError_t launch_mlp_pack(Ctx &c, cudaStream_t s)
{
    c.launches += 1;
    k_mlp_pack<<<(kMlpFragWords + 255) / 256, 256, 0, s>>>(c.mlp.w, c.mlp.frag);
    return cudaGetLastError();
}

cudaError_t launch_mlp_permute(Ctx &c, const unsigned *perm, int n, cudaStream_t s)
{
    const int g = (n + 255) / 256;
    c.launches += 2;
    k_mlp_gather<<<g, 256, 0, s>>>(perm, n, (int)c.capacity, c.mlp.tfeat, c.mlp.th,
                                   (float *)c.tmp);
    k_mlp_scatter_back<<<g, 256, 0, s>>>(n, (int)c.capacity, (const float *)c.tmp, c.mlp.tfeat,
                                         c.mlp.th);
    return cudaGetLastError();
}

cudaError_t launch_mlp_harvest(Ctx &c, const sph_particles &p, cudaStream_t s)
{
    const int n = (int)p.n;
    c.launches += 1;
    k_mlp_harvest<<<(n + 255) / 256, 256, 0, s>>>(n, (int)c.capacity, c.mlp.tfeat, c.mlp.th, p.h,
                                                  c.mlp.step++, (unsigned)c.mlp.stride,
                                                  (long long)c.mlp.cap, c.mlp.sx, c.mlp.sy,
                                                  c.mlp.scount);
    return cudaGetLastError();
}

int mlp_grad_blocks(long long batch)
{
    const long long nchunks = (batch + kMlpBlock - 1) / kMlpBlock;
    return (int)(nchunks < kMlpMaxBlocks ? nchunks : kMlpMaxBlocks);
}

cudaError_t launch_mlp_grad(Ctx &c, const float *sx, const float *sy, long long count,
                            long long batch, int random, unsigned long long seed, int iter,
                            cudaStream_t s)
{
    static bool attr_set[64] = {};
    const int dev = c.device & 63;
    if (!attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(MlpShared));
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    c.launches += 1;
    k_mlp_grad<<<mlp_grad_blocks(batch), kMlpBlock, sizeof(MlpShared), s>>>(
        c.mlp.w, sx, sy, count, batch, random, seed, iter, c.mlp.gpart);
    return cudaGetLastError();
}

cudaError_t launch_mlp_update(Ctx &c, long long batch, int adam, double lr, float *grad_out,
                              double *loss, cudaStream_t s)
{
    double lr_t = 0.0, eps_t = 1e-8;
    const double b1 = 0.9, b2 = 0.999;
    if (adam) {
        // mhat / (sqrt(vhat) + eps) = [m / (1 - b1^t)] / [sqrt(v) / sqrt(1 - b2^t) + eps]
        const int t = ++c.mlp.t;
        const double c1 = 1.0 - pow(b1, t), c2 = sqrt(1.0 - pow(b2, t));
        lr_t = lr * c2 / c1;
        eps_t = 1e-8 * c2;
    }
    c.launches += 1;
    k_mlp_update<<<(kMlpPart + 255) / 256, 256, 0, s>>>(c.mlp.gpart, mlp_grad_blocks(batch), batch,
                                                        adam, c.mlp.w, c.mlp.m, c.mlp.v, lr_t, b1,
                                                        b2, eps_t, grad_out, loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_infer(Ctx &c, const float *x, long long n, float *y, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    c.launches += 1;
    k_mlp_infer<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(c.mlp.frag, c.mlp.w, x, n, y);
    return cudaGetLastError();
}

}  // namespace sph
