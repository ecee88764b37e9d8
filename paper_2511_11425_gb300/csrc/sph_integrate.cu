// sph_integrate.cu -- kick-drift-kick with one global step per instance
// (Sec. 2.3.6) and the conserved totals.
//
//   closing kick   v_i = v_{i-1/2} + dt_old/2 a_i,      u_i likewise with du/dt
//   step choice    dt_new = dt_fixed, or min_i dt_i (Sec. 2.3.6 criteria)
//   opening kick   v_{i+1/2} = v_i + dt_new/2 a_i,     u likewise
//   drift          x_{i+1} = x_i + dt_new v_{i+1/2}, wrapped into periodic boxes
// du/dt is du/dt|H + du/dt|Pi (PdV form) or du/dt|Pi alone when u is moved
// along its adiabat after the density pass (entropy-conserving form).
// Everything here is FP64 per particle and memory-bound.
#include "sph_internal.cuh"
#include "sph_bits.h"

namespace sph {

// one thread per instance: dts[2k] = dt_old, dts[2k+1] = dt_new
__global__ void k_choose_dt(int ninst, double *dts, const unsigned *dtmin, double dt_fixed,
                            DevStatus *st)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ninst) return;
    double dt = dt_fixed > 0.0 ? dt_fixed : (double)__uint_as_float(dtmin[k]);
    if (!(dt > 0.0) || !isfinite(dt)) {
        raise_status(st, ST_NONFINITE, -1 - k);
        dt = 0.0;
    }
    dts[2 * k + 1] = dt;
}

// the new step becomes the old one, unless the step failed: then neither
// the state nor the step clock moves
__global__ void k_dt_shift(int ninst, double *dts, const DevStatus *st)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < ninst && st->code == 0) dts[2 * k] = dts[2 * k + 1];
}

// one particle's kicks and drift; h_next is the seed of the next density pass
// order-preserving integer key of a double: for non-NaN a, b,
// a < b  <=>  dkey(a) < dkey(b), except that -0 sorts just below +0 (IEEE 754
// binary64: sign-magnitude, so negative patterns are reflected)
__device__ __forceinline__ long long dkey(double d)
{
    const long long b = __double_as_longlong(d);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

__device__ __forceinline__ void kdk_particle(
    int i, const Inst *__restrict__ insts, const unsigned short *__restrict__ pinst, double *x,
    double *y, double *z, double *vx, double *vy, double *vz, double *u, float *h,
    const float *__restrict__ ax, const float *__restrict__ ay, const float *__restrict__ az,
    const float *__restrict__ dudt_h, const float *__restrict__ dudt_av, int energy_mode,
    const double *__restrict__ dts, float h_next, float *rho, const float4 *__restrict__ fth,
    const float *__restrict__ divv)
{
    const int k = pinst[i];
    const Inst &I = insts[k];
    const double dt_old = dts[2 * k], dt_new = dts[2 * k + 1];
    const double kick = 0.5 * (dt_old + dt_new);
    // FP32 -> FP64 on the integer pipes (exact; the FP64 pipe runs at 1/64
    // of the FP32 rate and carries the kick and drift themselves)
    double ud = bits::f2d(dudt_av[i]);
    if (energy_mode == SPH_ENERGY_PDV) ud += bits::f2d(dudt_h[i]);
    const double v0 = vx[i] + kick * bits::f2d(ax[i]);
    const double v1 = vy[i] + kick * bits::f2d(ay[i]);
    const double v2 = vz[i] + kick * bits::f2d(az[i]);
    vx[i] = v0;
    vy[i] = v1;
    vz[i] = v2;
    u[i] += kick * ud;
    // evolved density (mass conservation equation), kicked like u with the
    // rate -rho_pred div v of this step's force pass
    if (rho) rho[i] = (float)((double)rho[i] - kick * (double)fth[i].z * (double)divv[i]);
    double p[3] = {x[i] + dt_new * v0, y[i] + dt_new * v1, z[i] + dt_new * v2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // a particle moves far less than a box length per step: only one
        // that left [lo, hi) is wrapped.  The test compares order-preserving
        // integer keys of the IEEE 754 bit patterns (integer pipes; FP64
        // compares issue at the FP64 rate); a NaN lands in the wrap branch,
        // as with the FP64 compare, and -0 counts as below +0 (the wrap
        // then returns +0, the same value)
        const long long kp_ = dkey(p[a]);
        if (I.periodic[a] && !(kp_ >= dkey(I.lo[a]) && kp_ < dkey(I.hi[a]))) {
            double t = p[a] - I.lo[a];
            t -= I.Ld[a] * floor(t * I.invLd[a]);
            if (t >= I.Ld[a]) t -= I.Ld[a];
            if (t < 0.0) t = 0.0;
            p[a] = I.lo[a] + t;
        }
    }
    x[i] = p[0];
    y[i] = p[1];
    z[i] = p[2];
    h[i] = h_next;
}

// The smoothing length is advanced with the drift as the seed of the next
// density pass: the continuity equation gives rho(t + dt) ~ rho exp(-dt div v),
// and h ~ rho^(-1/3), so h <- h exp(dt div v / 3) (factor clamped to [1/2, 2]).
// CORR: the learned form adds the correction corr[i] (k_mlp_seed) to that
// exponent.
template <bool CORR>
__global__ void k_kdk(KParams kp, int n, const Inst *__restrict__ insts,
                      const unsigned short *__restrict__ pinst, double *x, double *y, double *z,
                      double *vx, double *vy, double *vz, double *u, float *h,
                      const float *__restrict__ ax, const float *__restrict__ ay,
                      const float *__restrict__ az, const float *__restrict__ dudt_h,
                      const float *__restrict__ dudt_av, const float *__restrict__ divv,
                      const double *__restrict__ dts, const float *__restrict__ corr,
                      float *rho_ev, const float4 *__restrict__ fth, const DevStatus *st)
{
    // an error raised earlier in the step leaves the state as it was
    if (st->code != 0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float e = bits::d2f(dts[2 * pinst[i] + 1]) * divv[i] * (1.f / 3.f);
    if (CORR) e += corr[i];
    const float f = expf(e);
    kdk_particle(i, insts, pinst, x, y, z, vx, vy, vz, u, h, ax, ay, az, dudt_h, dudt_av,
                 kp.energy_mode, dts, h[i] * fminf(fmaxf(f, 0.5f), 2.f), rho_ev, fth, divv);
}


// conserved totals per instance: grid (blocks, ninst); each block sums a
// fixed slice of its instance in a fixed tree order, then one block per
// instance folds the block partials in order (bit-identical from run to run)
constexpr int kConsThreads = 256;

// one particle into the running sums: momentum q = m v, then L += x × q,
// 2 E_kin += q·v and E_int += m u as fused multiply-adds (the factor 1/2 of
// E_kin is applied once, to the total)
__device__ __forceinline__ void cons_add(double acc[9], double mi, const double p[3],
                                         const double v[3], double u)
{
    const double q[3] = {mi * v[0], mi * v[1], mi * v[2]};
    acc[0] += mi;
    acc[1] += q[0];
    acc[2] += q[1];
    acc[3] += q[2];
    acc[4] = fma(p[1], q[2], fma(-p[2], q[1], acc[4]));
    acc[5] = fma(p[2], q[0], fma(-p[0], q[2], acc[5]));
    acc[6] = fma(p[0], q[1], fma(-p[1], q[0], acc[6]));
    acc[7] = fma(q[0], v[0], fma(q[1], v[1], fma(q[2], v[2], acc[7])));
    acc[8] = fma(mi, u, acc[8]);
}

// the block's nine partial sums in a fixed tree order, stored at `out`
__device__ __forceinline__ void cons_block_store(const double acc[9], double *out)
{
    __shared__ double sm[9][kConsThreads];
#pragma unroll
    for (int k = 0; k < 9; ++k) sm[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int o = kConsThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
#pragma unroll
            for (int k = 0; k < 9; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x < 9) out[threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void __launch_bounds__(kConsThreads) k_cons_partial(
    const Inst *__restrict__ insts, const double *__restrict__ x, const double *__restrict__ y,
    const double *__restrict__ z, const double *__restrict__ vx, const double *__restrict__ vy,
    const double *__restrict__ vz, const double *__restrict__ u, const float *__restrict__ m,
    double *part)
{
    const Inst &I = insts[blockIdx.y];
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const int b0 = I.off + blockIdx.x * kConsChunk, b1 = min(b0 + kConsChunk, I.off + I.n);
    for (int i = b0 + threadIdx.x; i < b1; i += kConsThreads) {
        const double p[3] = {x[i], y[i], z[i]}, v[3] = {vx[i], vy[i], vz[i]};
        cons_add(acc, (double)m[i], p, v, u[i]);
    }
    cons_block_store(acc, part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 9);
}

// nine warps per instance, one per total; each lane sums a fixed stride of
// the block partials and the warp folds the lanes in a fixed butterfly order
__global__ void k_cons_final(int nblocks, const double *part, double *out)
{
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (q >= 9) return;
    const double *pp = part + (size_t)blockIdx.x * nblocks * 9;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += pp[b * 9 + q];
    s = warp_sum(s);
    if (lane == 0) out[blockIdx.x * 9 + q] = q == 7 ? 0.5 * s : s;  // E_kin = (sum m v^2) / 2
}

cudaError_t launch_kdk(Ctx &c, const sph_particles &p, double dt_fixed, cudaStream_t s)
{
    const int n = (int)p.n;
    const int ni = c.kp.ninst;
    c.launches += 3;
    const int pr = prof_begin(c, s, SPH_PHASE_KDK);
    k_choose_dt<<<(ni + 127) / 128, 128, 0, s>>>(ni, c.dts, c.dtmin, dt_fixed, c.st);
    const bool corr = c.mlp.seed_mode == SPH_SEED_MLP;
    if (corr || c.mlp.record) {  // network inputs, records, corrections
        const cudaError_t e = launch_mlp_seed(c, p, s);
        if (e != cudaSuccess) return e;
    }
    const int g = (n + 255) / 256;
    if (corr)
        k_kdk<true><<<g, 256, 0, s>>>(c.kp, n, c.inst, c.pinst, p.x[0], p.x[1], p.x[2], p.v[0],
                                      p.v[1], p.v[2], p.u, p.h, p.a[0], p.a[1], p.a[2],
                                      p.dudt_h, p.dudt_av, p.divv, c.dts, c.mlp.corr,
                                      c.kp.evolved ? p.rho : nullptr, c.fth, c.st);
    else
        k_kdk<false><<<g, 256, 0, s>>>(c.kp, n, c.inst, c.pinst, p.x[0], p.x[1], p.x[2], p.v[0],
                                       p.v[1], p.v[2], p.u, p.h, p.a[0], p.a[1], p.a[2],
                                       p.dudt_h, p.dudt_av, p.divv, c.dts, nullptr,
                                       c.kp.evolved ? p.rho : nullptr, c.fth, c.st);
    k_dt_shift<<<(ni + 127) / 128, 128, 0, s>>>(ni, c.dts, c.st);
    prof_end(c, s, pr);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// hierarchical time steps (Sec. 2.3.6): substep `sub` of 2^R, length delta.
// An active particle (its period divides sub) closes its old step with the
// derivatives just computed (half its old period; none on the very first
// substep), picks its rung (ceil(log2(dt0 / dt_i)) clamped to [0, R], raised
// to the largest rung of its force partners less two; a lower rung only to
// one whose period divides sub, the lowest such) and opens the new step with
// half the new period.  Every particle drifts by delta; the seed of the next
// density pass is h exp(delta div v / 3) (factor clamped to [1/2, 2]).
// ---------------------------------------------------------------------------
__global__ void k_kdk_rungs(KParams kp, int n, const Inst *__restrict__ insts,
                            const unsigned short *__restrict__ pinst, double *x, double *y,
                            double *z, double *vx, double *vy, double *vz, double *u, float *h,
                            const float *__restrict__ ax, const float *__restrict__ ay,
                            const float *__restrict__ az, const float *__restrict__ dudt_h,
                            const float *__restrict__ dudt_av, const float *__restrict__ divv,
                            const float *__restrict__ dt_i, uint8_t *rung,
                            const int *__restrict__ rmax, RungArgs ra, const DevStatus *st)
{
    if (st->code != 0) return;  // a failed substep leaves the state as it was
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r_old = rung[i];
    double kick = 0.0;  // the closing and opening half periods of an active particle
    if (rung_active(ra.sub, ra.R, r_old)) {
        if (ra.started) kick = 0.5 * (double)(1 << (ra.R - r_old)) * ra.delta;
        // ceil(log2(dt0 / dt_i)) from the binary exponent (exact at powers of two)
        int e = 0;
        const double f = frexp(ra.dt0 / (double)dt_i[i], &e);
        int want = f == 0.5 ? e - 1 : e;
        want = max(want, rmax[i] - 2);
        want = min(max(want, 0), ra.R);
        int r_new = want;
        if (want < r_old) {  // a longer step only on a boundary of that step
            r_new = r_old;
            for (int r = want; r < r_old; ++r)
                if (rung_active(ra.sub, ra.R, r)) {
                    r_new = r;
                    break;
                }
        }
        rung[i] = (uint8_t)r_new;
        kick += 0.5 * (double)(1 << (ra.R - r_new)) * ra.delta;
    }
    const Inst &I = insts[pinst[i]];
    double ud = bits::f2d(dudt_av[i]);
    if (kp.energy_mode == SPH_ENERGY_PDV) ud += bits::f2d(dudt_h[i]);
    const double v0 = vx[i] + kick * bits::f2d(ax[i]);
    const double v1 = vy[i] + kick * bits::f2d(ay[i]);
    const double v2 = vz[i] + kick * bits::f2d(az[i]);
    vx[i] = v0;
    vy[i] = v1;
    vz[i] = v2;
    u[i] += kick * ud;
    double p[3] = {x[i] + ra.delta * v0, y[i] + ra.delta * v1, z[i] + ra.delta * v2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (I.periodic[a] && !(p[a] >= I.lo[a] && p[a] < I.hi[a])) {
            double t = p[a] - I.lo[a];
            t -= I.Ld[a] * floor(t * I.invLd[a]);
            if (t >= I.Ld[a]) t -= I.Ld[a];
            if (t < 0.0) t = 0.0;
            p[a] = I.lo[a] + t;
        }
    }
    x[i] = p[0];
    y[i] = p[1];
    z[i] = p[2];
    const float g = expf((float)ra.delta * divv[i] * (1.f / 3.f));
    h[i] = h[i] * fminf(fmaxf(g, 0.5f), 2.f);
}

__global__ void k_rung_gather(const unsigned *__restrict__ perm, int n, const uint8_t *rung,
                              int *tmp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) tmp[i] = rung[perm[i]];
}

__global__ void k_rung_copyback(int n, const int *__restrict__ tmp, uint8_t *rung)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rung[i] = (uint8_t)tmp[i];
}

cudaError_t launch_rung_permute(Ctx &c, const unsigned *perm, int n, cudaStream_t s)
{
    c.launches += 2;
    k_rung_gather<<<(n + 255) / 256, 256, 0, s>>>(perm, n, c.rung, c.rmax);
    k_rung_copyback<<<(n + 255) / 256, 256, 0, s>>>(n, c.rmax, c.rung);
    return cudaGetLastError();
}

cudaError_t launch_kdk_rungs(Ctx &c, const sph_particles &p, const RungArgs &ra, cudaStream_t s)
{
    const int n = (int)p.n;
    c.launches += 1;
    const int pr = prof_begin(c, s, SPH_PHASE_KDK);
    k_kdk_rungs<<<(n + 255) / 256, 256, 0, s>>>(c.kp, n, c.inst, c.pinst, p.x[0], p.x[1], p.x[2],
                                                p.v[0], p.v[1], p.v[2], p.u, p.h, p.a[0], p.a[1],
                                                p.a[2], p.dudt_h, p.dudt_av, p.divv, p.dt_i, c.rung,
                                                c.rmax, ra, c.st);
    prof_end(c, s, pr);
    return cudaGetLastError();
}

cudaError_t launch_conserved(Ctx &c, const sph_particles &p, cudaStream_t s)
{
    const int nb = c.cons_blocks > 0 ? c.cons_blocks : 1;
    c.launches += 2;
    const int pr = prof_begin(c, s, SPH_PHASE_CONSERVED);
    k_cons_partial<<<dim3(nb, c.kp.ninst), kConsThreads, 0, s>>>(
            c.inst, p.x[0], p.x[1], p.x[2], p.v[0], p.v[1], p.v[2], p.u, p.m, c.cons_part);
    k_cons_final<<<c.kp.ninst, 288, 0, s>>>(nb, c.cons_part, c.cons_out);
    prof_end(c, s, pr);
    return cudaGetLastError();
}

}  // namespace sph
