// sph_forces.cu -- time derivatives (Sec. 2.3.5) and time-step limits (Sec. 2.3.6).
//
// For every unordered pair (i, j) with r_ij < max(h_i, h_j), evaluated ONCE:
//   F_i = dW_ij(h_i)/dr / r = sigma h_i^-5 (w'(q_i)/q_i)     (grad_i W_ij(h_i) = r_ij F_i)
//   pressure:  a_i -= m_j (A_i F_i + A_j F_j) r_ij,  a_j += m_i (A_i F_i + A_j F_j) r_ij,
//              A = P / (Omega rho^2)                               (momentum equation)
//   S_i += m_j (v_ij.r_ij) F_i,  S_j += m_i (v_ij.r_ij) F_j          (S = sum m v_ij.grad W)
//   viscosity, only for v_ij.r_ij < 0:
//              mu = hbar (v_ij.r_ij)/(r^2 + eps hbar^2),
//              Pi = (-alpha cbar mu + beta mu^2)/rhobar,  Fbar = (F_i + F_j)/2
//              a_i -= m_j Pi Fbar r_ij,  a_j += m_i Pi Fbar r_ij
//              du_i|Pi += m_j Pi (v_ij.r_ij) Fbar / 2,  du_j|Pi += m_i Pi (v_ij.r_ij) Fbar / 2
//   Courant:   max_j |min(0, mu_ij)| for both particles
// and afterwards (finalize)
//   du/dt|H = A_i S_i (PdV equation),  div v = -S_i/(Omega_i rho_i),
//   dt_i = min(eta_a sqrt(h_i/|a_i|), eta_C h_i / ((1+0.6 alpha) c_i + 0.6 beta max|mu|)).
//
// GPU mapping: one warp per sink bucket A, lane = sink particle.  The list
// holds source buckets B >= A whose bounds pass the gather or scatter test
// (Sec. 2.3.2); source particles are culled per particle, compacted into a
// 128-entry shared-memory chunk, and each lane marks its hits in a 128-bit
// mask.  A chunk then takes ceil(hits / 32) rounds: every lane evaluates its
// own hits up to that count and the surplus of the busier lanes is dealt to
// the idle ones (force_chunk).  Contributions to a lane's own sink stay in
// registers; the equal and opposite contribution to the source, and the sink
// side of a dealt pair, go straight to L2 as fire-and-forget reductions (the
// SM does not wait): a xyz and du/dt|Pi as one red.global.add.v4.f32, S as
// one red.global.add.f64 (which measured as fast as keeping S in the FP32
// vector: the reductions are not the bottleneck).  j > i is required inside
// bucket A, so every pair is computed exactly once.
//
// Precision.  Pair arithmetic is FP32 on positions relative to the sink
// bucket's origin.  S_i is a sum whose terms cancel (across a shear layer
// v_ij.r_ij changes sign with the geometry and the sum is a small fraction of
// the terms' magnitudes), so its terms are computed without the two roundings
// that dominate there: the separations are exact integer differences of
// fixed-point positions (units qx = q 2^-11 relative to the bucket origins),
// converted to FP32 once, and the kernel factor 1 - q comes from the exact
// integer N = h^2 - r^2 as (N qx^2 / h^2) / (1 + q) instead of from a rounded
// q = r/h.  S is accumulated with a Kahan sum per term on the sink side of a
// lane's own pairs and in FP64 through L2 otherwise (the accelerations per
// 128-candidate chunk, the chunks' partial sums added in FP32).  Instances whose buckets or h outgrow the
// fixed-point range (tiny open boxes), and sink buckets whose pairs need a
// periodic wrap of their own, use FP32 separations and q throughout.
#include "sph_internal.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// predictor + EOS (Sec. 2.3.6 step 2, Sec. 2.3.1)
// ---------------------------------------------------------------------------
__global__ void k_predict(KParams kp, int n, const Inst *__restrict__ insts,
                          const unsigned short *__restrict__ pinst, const double *__restrict__ vx,
                          const double *__restrict__ vy, const double *__restrict__ vz,
                          const double *__restrict__ u, const float *__restrict__ ax,
                          const float *__restrict__ ay, const float *__restrict__ az,
                          const float *__restrict__ dudt_h, const float *__restrict__ dudt_av,
                          const float *__restrict__ h, const float *__restrict__ rho,
                          const float *__restrict__ omega, const float4 *__restrict__ pm,
                          const double *__restrict__ dts, float4 *fpos, float4 *fvel, float4 *fth,
                          int4 *ipos, float4 *acc, double *accS, unsigned *mumax, unsigned *dtmin,
                          double4_16a *fveld, double4_16a *fthd, double4_16a *acc64,
                          const float *__restrict__ divv_old, const uint8_t *__restrict__ mat,
                          float2 *ic_pt, RungArgs ra, DevStatus *st)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kp.ninst) dtmin[i] = 0x7f800000u;  // +inf
    if (i >= n) return;
    const int k = pinst[i];
    const Inst &I = insts[k];
    const float gamma = I.gamma;
    // time from the half-step state (v, u) to now: half the old step, or in
    // a hierarchical step the time since the particle's last boundary (its
    // whole period when it is active now) less half its period
    double hdt = 0.5 * dts[2 * k];
    if (ra.rung) {
        const int P = 1 << (ra.R - (int)ra.rung[i]);
        const int phi = ra.sub & (P - 1);
        hdt = ra.started ? ((double)(phi == 0 ? P : phi) - 0.5 * (double)P) * ra.delta : 0.0;
        ra.rmax[i] = -1;
    }
    double v[3] = {vx[i], vy[i], vz[i]};
    double uu = u[i];
    if (hdt != 0.0) {
        v[0] += hdt * (double)ax[i];
        v[1] += hdt * (double)ay[i];
        v[2] += hdt * (double)az[i];
        double ud = (double)dudt_av[i];
        if (kp.energy_mode == SPH_ENERGY_PDV) ud += (double)dudt_h[i];
        uu += hdt * ud;
    }
    float r = rho[i], om = omega[i], hi = h[i];
    // evolved density: predicted like u, with the rate -rho div v of the
    // last force pass
    if (kp.evolved && hdt > 0.0) r = (float)((double)r * (1.0 - hdt * (double)divv_old[i]));
    float P = (gamma - 1.f) * r * (float)uu;
    float c = sqrtf(gamma * P / r);
    float A = P / (om * r * r);
    if (!(isfinite(A) && isfinite(c) && uu >= 0.0)) raise_status(st, ST_NONFINITE, i);
    if (fveld) {  // FP64 form: the same records in FP64
        const double rd = (double)r, od = (double)om, gd = (double)gamma;
        const double Pd = (gd - 1.0) * rd * uu;
        fveld[i] = make_double4_16a(v[0], v[1], v[2], (double)pm[i].w);
        fthd[i] = make_double4_16a(Pd / (od * rd * rd), sqrt(gd * Pd / rd), rd, od);
        acc64[i] = make_double4_16a(0.0, 0.0, 0.0, 0.0);
    }
    float4 q = pm[i];
    fpos[i] = make_float4(q.x, q.y, q.z, hi);
    fvel[i] = make_float4((float)v[0], (float)v[1], (float)v[2], q.w);
    fth[i] = make_float4(A, c, r, om);
    // interface correction: pressure and temperature (T = (gamma-1) u / R
    // of the particle's material) for the correction pass
    if (ic_pt) ic_pt[i] = make_float2(P, (gamma - 1.f) * (float)uu / I.r_gas[mat[i] & 3]);
    // h in fixed-point units (h < fix_lim whenever the force kernel uses it)
    reinterpret_cast<int *>(ipos + i)[3] = __float2int_rn(fminf(hi, I.fix_lim) * I.inv_qx);
    acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    accS[i] = 0.0;
    mumax[i] = 0u;
}

// ---------------------------------------------------------------------------
// pair-symmetric force kernel
// ---------------------------------------------------------------------------
#ifndef SPH_FORCE_BLOCKS_PER_SM
#define SPH_FORCE_BLOCKS_PER_SM 5
#endif
constexpr int kForceBlocksPerSM = SPH_FORCE_BLOCKS_PER_SM;


// per-lane sink state kept in registers: what the candidate masks need, the
// sink-side sums and the counters
struct SinkState {
    float px, py, pz, h2;              // position in the sink frame, h^2
    int rg, rmx;                       // hierarchical steps: rung, largest partner rung
    float ax, ay, az;                  // sums of the chunks' partial sums
    Kahan S;
    float du, mumax;
    unsigned pairs, av;
};

// per-warp shared-memory copy of the sink bucket: the pair loop reads the
// sink of each pair from here, since a lane may evaluate a pair of another
// lane's sink (load balancing, force_chunk)
struct SinkStage {
    union {
        int4 ipos[32];   // fixed-point path: position (units qx) and h
        float4 pos[32];  // FP32 path: position in the sink frame
    };
    float4 vel[32];  // predicted velocity, m
    float4 th[32];   // A = P/(Omega rho^2), c, rho, h
    float2 ih[32];   // 1/h, sigma h^-5
};

// per-warp shared-memory stage of one chunk of source candidates
struct ForceStage {
    float4 pos[kChunk];  // position in the sink frame, h^2
    float4 vel[kChunk];  // predicted velocity, m
    float4 th[kChunk];   // A = P/(Omega rho^2), c, rho, h
    int4 ipos[kChunk];   // fixed-point position in the sink frame, h (units qx)
    float ih[kChunk];    // 1/h, correctly rounded (once per staged source)
    int idx[kChunk];
};

template <bool WRAP>
__device__ __forceinline__ void sep3(const PBox &bx, float px, float py, float pz, float4 q,
                                     float &dx, float &dy, float &dz)
{
    dx = px - q.x;
    dy = py - q.y;
    dz = pz - q.z;
    if (WRAP) {
        if (bx.per[0]) dx = wrapf(dx, bx.L[0], bx.invL[0]);
        if (bx.per[1]) dy = wrapf(dy, bx.L[1], bx.invL[1]);
        if (bx.per[2]) dz = wrapf(dz, bx.L[2], bx.invL[2]);
    }
}

// fire-and-forget reductions of the pair loop.  Nothing in the force kernel
// reads what they write, so they carry no compiler memory barrier and the
// next pair's shared-memory loads may be scheduled across them.
__device__ __forceinline__ void red_v4_nb(float4 *addr, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b),
                 "f"(c), "f"(d));
}
__device__ __forceinline__ void red_f64_nb(double *addr, double a)
{
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(addr), "d"(a));
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(kFull, v, d);
        if (lane >= d) v += t;
    }
    return v;
}

// position (0..127) of the q-th set bit (q from 0) of the 128-bit mask
// a0 | a1 << 32 | a2 << 64 | a3 << 96; q < popcount of the mask
__device__ __forceinline__ int select_bit128(unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                             int q)
{
    const int c0 = __popc(a0), c1 = __popc(a1), c2 = __popc(a2);
    int base = 0;
    unsigned x = a0;
    if (q >= c0) {
        q -= c0;
        base = 32;
        x = a1;
        if (q >= c1) {
            q -= c1;
            base = 64;
            x = a2;
            if (q >= c2) {
                q -= c2;
                base = 96;
                x = a3;
            }
        }
    }
    int c = __popc(x & 0xffffu);
    if (q >= c) { q -= c; x >>= 16; base += 16; }
    c = __popc(x & 0xffu);
    if (q >= c) { q -= c; x >>= 8; base += 8; }
    c = __popc(x & 0xfu);
    if (q >= c) { q -= c; x >>= 4; base += 4; }
    c = __popc(x & 0x3u);
    if (q >= c) { q -= c; x >>= 2; base += 2; }
    if (q >= (int)(x & 1u)) base += 1;
    return base;
}

// viscosity parameters and fixed-point quantum of the sink's instance
struct Visc {
    float alpha, beta, eps_av, qx, qx2;
};

// One staged chunk of candidates against the 32 sinks.
//
// SELF: the chunk holds the sink bucket's own particles, where only j > i
// counts (every other source bucket lies after the sink bucket, so all its
// particles do).  FIX: separations and 1 - q from the fixed-point positions.
//
// Load balance.  Lane l's hit mask holds c_l pairs; evaluated lane by lane
// the warp would take max_l c_l rounds, about 2.4 times the mean on a
// lattice.  Instead the chunk takes m = ceil(T / 32) rounds (T = sum c_l):
// lane l evaluates its first min(c_l, m) hits itself (sink side summed in
// registers) and the surplus hits of the lanes with c_l > m are dealt, in
// lane order, to the free rounds of the lanes with c_l < m; a dealt pair
// sends both of its sides to L2 as reductions.  RUNG keeps the lane-by-lane
// loop (the rung limiter tracks each sink's partners in registers).
template <class K, bool WRAP, bool SELF, bool FIX, bool RUNG>
__device__ __forceinline__ void force_chunk(const PBox &bx, const Visc &vp, ForceStage &S,
                                            const SinkStage &Q, int c, SinkState &s, bool valid,
                                            int lane, int i0, float4 *acc, double *accS,
                                            unsigned *mumax, const RungArgs &ra)
{
    const int nwords = (c + 31) >> 5;
    for (int k = c + lane; k < 32 * nwords; k += 32) {
        S.pos[k] = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
        S.idx[k] = -1;
    }
    __syncwarp();
    // hit masks: r < max(h_i, h_j) (and j > i in the own bucket): each
    // unordered pair once
    unsigned w0 = 0u, w1 = 0u, w2 = 0u, w3 = 0u;
    if (valid) {
#pragma unroll 1
        for (int ww = 0; ww < nwords; ++ww) {
            unsigned mw = 0u;
#pragma unroll
            for (int b = 31; b >= 0; --b) {  // bit b <- hit of candidate 32 ww + b
                const float4 q = S.pos[32 * ww + b];
                float dx, dy, dz;
                sep3<WRAP>(bx, s.px, s.py, s.pz, q, dx, dy, dz);
                float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                unsigned hit = __float_as_uint(r2 - fmaxf(s.h2, q.w)) >> 31;
                if (SELF) hit &= S.idx[32 * ww + b] > i0 + lane ? 1u : 0u;
                mw = mw * 2u + hit;
            }
            if (ww == 0) w0 = mw; else if (ww == 1) w1 = mw; else if (ww == 2) w2 = mw; else w3 = mw;
        }
    }
    unsigned long long m0 = (unsigned long long)w0 | ((unsigned long long)w1 << 32);
    unsigned long long m1 = (unsigned long long)w2 | ((unsigned long long)w3 << 32);
    float sax = 0.f, say = 0.f, saz = 0.f;
    // one pair (sink of lane o, candidate k): every term, no side effects
    struct PairTerms {
        float dx, dy, dz, cm, Si, mj, du, mneg, cs, Sj, du_j;
        int jj;
        bool app;
    };
    auto pair_terms = [&](int k, int o) -> PairTerms {
        PairTerms t;
        const float4 vi = Q.vel[o];
        const float4 thi = Q.th[o];  // A, c, rho, h
        const float2 ii = Q.ih[o];   // 1/h, sigma h^-5
        const float4 vj = S.vel[k];
        const float4 tj = S.th[k];
        const float hj = tj.w, ihj = S.ih[k];
        const float ihj2 = ihj * ihj;
        float dx, dy, dz, Fi, Fj, r2;
        if (FIX) {
            // exact integer separation and N = h^2 - r^2 (units qx), each
            // converted to FP32 with one rounding
            const int4 pi = Q.ipos[o];
            const int4 p = S.ipos[k];
            const int ex = (int)((unsigned)pi.x - (unsigned)p.x);
            const int ey = (int)((unsigned)pi.y - (unsigned)p.y);
            const int ez = (int)((unsigned)pi.z - (unsigned)p.z);
            const long long r2q = (long long)ex * ex + (long long)ey * ey + (long long)ez * ez;
            const long long ni = (long long)pi.w * pi.w - r2q;
            const long long nj = (long long)p.w * p.w - r2q;
            dx = (float)ex * vp.qx;
            dy = (float)ey * vp.qx;
            dz = (float)ez * vp.qx;
            r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float r = r2 * rsqrtf(fmaxf(r2, 1e-37f));
            const float qi = r * ii.x, qj = r * ihj;
            // 1 - q = (1 - q^2) / (1 + q) with 1 - q^2 = N qx^2 / h^2
            const float ti = __fdividef((float)ni * (vp.qx2 * ii.x * ii.x), 1.f + qi);
            const float tj_ = __fdividef((float)nj * (vp.qx2 * ihj2), 1.f + qj);
            Fi = ni > 0 ? ii.y * K::dwqt(qi, ti) : 0.f;
            Fj = nj > 0 ? K::sigma * ihj2 * ihj2 * ihj * K::dwqt(qj, tj_) : 0.f;
        } else {
            const float4 pi = Q.pos[o];
            const float4 q = S.pos[k];
            sep3<WRAP>(bx, pi.x, pi.y, pi.z, q, dx, dy, dz);
            r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float r = r2 * rsqrtf(fmaxf(r2, 1e-37f));
            const float qi = r * ii.x, qj = r * ihj;
            Fi = qi < 1.f ? ii.y * K::dwq(qi) : 0.f;
            Fj = qj < 1.f ? K::sigma * ihj2 * ihj2 * ihj * K::dwq(qj) : 0.f;
        }
        const float wx = vi.x - vj.x, wy = vi.y - vj.y, wz = vi.z - vj.z;
        const float vr = fmaf(wx, dx, fmaf(wy, dy, wz * dz));
        // viscosity, evaluated for every pair and switched by v_ij.r_ij < 0
        t.app = vr < 0.f;
        const float hb = 0.5f * (thi.w + hj), cb = 0.5f * (thi.y + tj.y),
                    rb = 0.5f * (thi.z + tj.z);
        // one reciprocal for mu's denominator and rhobar
        const float den = fmaf(vp.eps_av * hb, hb, r2);
        const float rdr = __fdividef(1.f, den * rb);
        const float mu = hb * vr * (rb * rdr);
        const float Pi = t.app ? fmaf(-vp.alpha * cb, mu, vp.beta * mu * mu) * (den * rdr) : 0.f;
        const float Fb = 0.5f * (Fi + Fj);
        const float coef = fmaf(thi.x, Fi, fmaf(tj.x, Fj, Pi * Fb));
        const float du = 0.5f * Pi * vr * Fb;
        t.mneg = t.app ? -mu : 0.f;
        t.dx = dx;
        t.dy = dy;
        t.dz = dz;
        t.cm = coef * vj.w;
        t.Si = vj.w * vr * Fi;
        t.mj = vj.w;
        t.du = du;
        t.cs = coef * vi.w;
        t.Sj = vi.w * vr * Fj;
        t.du_j = vi.w * du;
        t.jj = S.idx[k];
        return t;
    };
    // the source side of a pair: straight into global memory (L2 reductions)
    auto apply_far = [&](const PairTerms &t) {
        red_v4_nb(&acc[t.jj], t.cs * t.dx, t.cs * t.dy, t.cs * t.dz, t.du_j);
        red_f64_nb(&accS[t.jj], (double)t.Sj);
        if (t.app) {
            atomicMax(&mumax[t.jj], __float_as_uint(t.mneg));
            ++s.av;
        }
        ++s.pairs;
    };
    // the sink side of a lane's own pair: registers
    auto apply_own = [&](const PairTerms &t) {
        sax = fmaf(-t.cm, t.dx, sax);
        say = fmaf(-t.cm, t.dy, say);
        saz = fmaf(-t.cm, t.dz, saz);
        s.S.add(t.Si);
        s.du = fmaf(t.mj, t.du, s.du);
        s.mumax = fmaxf(s.mumax, t.mneg);
    };
    // lowest pending hit, without a branch (lanes differ in which half is
    // empty)
    auto next = [&]() -> int {
        const bool lo = m0 != 0ull;
        const unsigned long long w = lo ? m0 : m1;
        const int k = __ffsll((long long)w) - 1 + (lo ? 0 : 64);
        const unsigned long long w2 = w & (w - 1ull);
        m0 = lo ? w2 : m0;
        m1 = lo ? m1 : w2;
        return k;
    };
    if (RUNG) {
        while (m0 | m1) {
            const PairTerms t = pair_terms(next(), lane);
            apply_own(t);
            apply_far(t);
            // the rung limiter needs each particle's largest partner rung
            const int rj = ra.rung[t.jj];
            s.rmx = max(s.rmx, rj);
            if (rung_active(ra.sub, ra.R, rj)) atomicMax(&ra.rmax[t.jj], s.rg);
        }
    } else {
        const int cnt = __popcll(m0) + __popcll(m1);
        const int T = __reduce_add_sync(kFull, (unsigned)cnt);
        const int m = (T + 31) >> 5;               // rounds of the chunk
        const int cmin = (int)__reduce_min_sync(kFull, (unsigned)cnt);
        const int sur = max(cnt - m, 0), fre = max(m - cnt, 0);
        const int sex = warp_incl_scan(sur, lane) - sur;   // first surplus index of the lane
        const int fex = warp_incl_scan(fre, lane) - fre;   // first free slot of the lane
        const int stot = __shfl_sync(kFull, sex + sur, 31);
        for (int r = 0; r < m; ++r) {
            const bool own = r < cnt;
            int k = own ? next() : 0;
            int o = lane;
            bool act = own;
            if (r >= cmin && stot > 0) {  // warp-uniform: some lane has a free round
                // surplus index u of this lane's free round, its donor d (the
                // last lane whose surplus starts at or before u) and the
                // donor's pending hits (it has taken ranks 0..r itself)
                const int u = fex + (r - cnt);
                int d = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int sd = __shfl_sync(kFull, sex, d + step);
                    if (sd <= u) d += step;
                }
                const int sd = __shfl_sync(kFull, sex, d);
                const unsigned a0 = __shfl_sync(kFull, (unsigned)m0, d);
                const unsigned a1 = __shfl_sync(kFull, (unsigned)(m0 >> 32), d);
                const unsigned a2 = __shfl_sync(kFull, (unsigned)m1, d);
                const unsigned a3 = __shfl_sync(kFull, (unsigned)(m1 >> 32), d);
                if (!own && u < stot) {
                    k = select_bit128(a0, a1, a2, a3, m + (u - sd) - (r + 1));
                    o = d;
                    act = true;
                }
            }
            if (act) {
                const PairTerms t = pair_terms(k, o);
                if (o == lane) {
                    apply_own(t);
                } else {  // a dealt pair: the donor's sink side to L2 as well
                    const int io = i0 + o;
                    red_v4_nb(&acc[io], -t.cm * t.dx, -t.cm * t.dy, -t.cm * t.dz, t.mj * t.du);
                    red_f64_nb(&accS[io], (double)t.Si);
                    if (t.app) atomicMax(&mumax[io], __float_as_uint(t.mneg));
                }
                apply_far(t);
            }
        }
    }
    s.ax += sax;
    s.ay += say;
    s.az += saz;
    __syncwarp();
}

struct SinkBounds {
    float cen[3], gc[3], gr[3], bc[3], br[3];
    float gR2;
};

template <class K, bool WRAP, bool FIX, bool RUNG>
__device__ __forceinline__ void force_bucket(const KParams &kp, const Inst &I, const PBox &bx,
                                             const Visc &vp, int A, int lane, ForceStage &S,
                                             const SinkStage &Q, SinkState &s, bool valid,
                                             const SinkBounds sb,
                                             const int *__restrict__ bstart,
                                             const float4 *__restrict__ fpos,
                                             const float4 *__restrict__ fvel,
                                             const float4 *__restrict__ fth,
                                             const int4 *__restrict__ ipos,
                                             const unsigned *__restrict__ list_cnt,
                                             const unsigned *__restrict__ list_off,
                                             const unsigned *__restrict__ list,
                                             const int *__restrict__ origin,
                                             const float4 *__restrict__ node, float4 *acc,
                                             double *accS, unsigned *mumax,
                                             unsigned &cands, const RungArgs &ra)
{
    const unsigned lt = (1u << lane) - 1u;
    // Filter the group's list for this bucket (Sec. 2.3.2 tests with the
    // bucket's own bounds): source bucket B >= A whose cell bound meets the
    // sink box-of-balls (gather) or whose box-of-balls meets the sink cell
    // bound (scatter).  Lane w keeps the bits of entries 32w .. 32w+31.
    // Lists longer than one 1024-entry segment (overflow arena) are filtered
    // and processed segment by segment.
    const int g = group_of(I, A);
    const unsigned nl = list_cnt[g];
    const unsigned *__restrict__ gl = list + list_off[g];
    // bits of list entries 32w .. 32w+31 (the sink leaf's bounds are loaded
    // per call, not kept live across the pair loop)
    auto filter_word = [&](unsigned w) -> unsigned {
        const size_t ka = leaf_of(I, A);
        const float4 sb0 = node[4 * ka], sb1 = node[4 * ka + 1];
        const float4 so0 = node[4 * ka + 2], so1 = node[4 * ka + 3];
        const unsigned e = 32 * w + lane;
        bool acc_ = false;
        if (e < nl) {
            const unsigned B = gl[e];
            const size_t k = leaf_of(I, (int)B);
            if ((int)B >= A) {
                const float4 b0 = node[4 * k], b1 = node[4 * k + 1];
                acc_ = ovl(so0.x, so1.x, b0.x, b1.x, bx.per[0], bx.L[0], bx.invL[0]) &&
                       ovl(so0.y, so1.y, b0.y, b1.y, bx.per[1], bx.L[1], bx.invL[1]) &&
                       ovl(so0.z, so1.z, b0.z, b1.z, bx.per[2], bx.L[2], bx.invL[2]);
                if (!acc_) {
                    const float4 o0 = node[4 * k + 2], o1 = node[4 * k + 3];
                    acc_ = ovl(sb0.x, sb1.x, o0.x, o1.x, bx.per[0], bx.L[0], bx.invL[0]) &&
                           ovl(sb0.y, sb1.y, o0.y, o1.y, bx.per[1], bx.L[1], bx.invL[1]) &&
                           ovl(sb0.z, sb1.z, o0.z, o1.z, bx.per[2], bx.L[2], bx.invL[2]);
                }
            }
        }
        return __ballot_sync(kFull, acc_);
    };
    unsigned myword = 0u;
    for (unsigned w = 0; 32 * w < nl && w < 32; ++w) {
        const unsigned bal = filter_word(w);
        if (lane == (int)w) myword = bal;
    }
    // what staging needs of a source bucket: its first particle and length
    // and its origin minus the sink bucket's (grid points)
    struct SrcRec {
        int j0, len, dk[3];
    };
    auto src_rec = [&](int B) -> SrcRec {
        SrcRec r;
#pragma unroll
        for (int a = 0; a < 3; ++a) r.dk[a] = origin[a * kp.nb + B] - origin[a * kp.nb + A];
        r.j0 = bstart[B];
        r.len = bucket_len(bstart, B);
        return r;
    };
    // stage the culled particles of the source bucket r after the c staged ones
    auto stage = [&](const SrcRec &r, int c) -> int {
        const int j = r.j0 + lane;
        const bool vj = lane < r.len;
        const float4 q = vj ? fpos[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        // the other records are loaded with the position, before the cull
        // decides, so that their L2 latency overlaps the first one
        float4 t4 = make_float4(0.f, 0.f, 0.f, 0.f), v4 = t4;
        int4 p4 = make_int4(0, 0, 0, 0);
        if (vj) {
            t4 = fth[j];
            v4 = fvel[j];
            if (FIX) p4 = ipos[j];
        }
        // origin offset in the sink frame (nearest periodic image), as FP32
        // and, for the fixed-point path, in units of qx modulo 2^32
        float d[3];
        unsigned o3[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float f = (float)r.dk[a] * I.qf;
            int nimg = 0;
            if (bx.per[a]) {
                nimg = (int)rintf(f * bx.invL[a]);
                f -= bx.L[a] * (float)nimg;
            }
            d[a] = f;
            o3[a] = ((unsigned)r.dk[a] << kFixShift) - (unsigned)nimg * I.LQ[a];
        }
        float sp[3] = {d[0] + q.x, d[1] + q.y, d[2] + q.z};
        // gather: inside the sink's box of balls and ball of balls;
        // scatter: the source's own ball reaches the sink cell bound
        bool gbox = true;
        float dg2 = 0.f, dd = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float dg = sp[a] - sb.gc[a];
            float dc = sp[a] - sb.bc[a];
            if (WRAP && bx.per[a]) {
                sp[a] -= bx.L[a] * rintf((sp[a] - sb.cen[a]) * bx.invL[a]);
                dg = wrapf(dg, bx.L[a], bx.invL[a]);
                dc = wrapf(dc, bx.L[a], bx.invL[a]);
            }
            gbox = gbox && fabsf(dg) <= sb.gr[a];
            dg2 = fmaf(dg, dg, dg2);
            float o = fmaxf(fabsf(dc) - sb.br[a], 0.f);
            dd = fmaf(o, o, dd);
        }
        const bool in = vj && ((gbox && dg2 <= sb.gR2) || dd < q.w * q.w);
        const unsigned bal = __ballot_sync(kFull, in);
        if (in) {
            const int pos = c + __popc(bal & lt);
            const float4 t = t4;
            S.pos[pos] = make_float4(sp[0], sp[1], sp[2], q.w * q.w);
            S.vel[pos] = v4;
            S.th[pos] = make_float4(t.x, t.y, t.z, q.w);
            S.ih[pos] = __frcp_rn(q.w);
            S.idx[pos] = j;
            if (FIX) {
                // the source in the sink frame: its fixed-point position plus
                // the origin offset, modulo 2^32
                const int4 p = p4;
                S.ipos[pos] = make_int4((int)((unsigned)p.x + o3[0]), (int)((unsigned)p.y + o3[1]),
                                        (int)((unsigned)p.z + o3[2]), p.w);
            }
        }
        c += __popc(bal);
        return c;
    };
    // the sink bucket itself (the only source bucket needing j > i)
    int c = stage(src_rec(A), 0);
    if (c > 0) {
        __syncwarp();
        cands += c;
        force_chunk<K, WRAP, true, FIX, RUNG>(bx, vp, S, Q, c, s, valid, lane, bstart[A], acc, accS, mumax,
                                               ra);
        c = 0;
    }
    const unsigned nwords = (nl + 31) / 32;
    for (unsigned w = 0; w < nwords; ++w) {
      // words past the first 32 (long lists in the overflow arena) are
      // filtered when reached
      unsigned mw = w < 32 ? __shfl_sync(kFull, myword, w) : filter_word(w);
      if (!mw) continue;
      // the records of this word's accepted entries, one per lane, fetched
      // together (one round of dependent loads per word, not per entry)
      SrcRec mine{};
      int myB = -1;
      if ((mw >> lane) & 1u) {
          myB = (int)gl[32 * w + lane];
          if (myB != A) mine = src_rec(myB);
      }
      while (mw) {
        const int l = __ffs(mw) - 1;
        mw &= mw - 1u;
        if (__shfl_sync(kFull, myB, l) == A) continue;
        SrcRec r;
        r.j0 = __shfl_sync(kFull, mine.j0, l);
        r.len = __shfl_sync(kFull, mine.len, l);
#pragma unroll
        for (int a = 0; a < 3; ++a) r.dk[a] = __shfl_sync(kFull, mine.dk[a], l);
        c = stage(r, c);
        if (c > kChunk - 32) {
            __syncwarp();
            cands += c;
            force_chunk<K, WRAP, false, FIX, RUNG>(bx, vp, S, Q, c, s, valid, lane, bstart[A], acc, accS,
                                                mumax, ra);
            c = 0;
        }
      }
    }
    if (c > 0) {
        __syncwarp();
        cands += c;
        force_chunk<K, WRAP, false, FIX, RUNG>(bx, vp, S, Q, c, s, valid, lane, bstart[A], acc, accS,
                                                mumax, ra);
    }
}

// 5 blocks of 4 warps per SM (96 registers; the fixed-point pair path spills
// a few values; 43 KB of shared memory per block): measured faster than 4
// blocks without spills
// one sink bucket A (one warp)
template <class K, bool RUNG>
__device__ __forceinline__ void force_sink(const KParams &kp, const Inst *__restrict__ insts,
                                           const int *__restrict__ bstart,
                                           const int *__restrict__ binst,
                                           const float4 *__restrict__ fpos,
                                           const float4 *__restrict__ fvel,
                                           const float4 *__restrict__ fth,
                                           const int4 *__restrict__ ipos,
                                           const unsigned *__restrict__ list_cnt,
                                           const unsigned *__restrict__ list_off,
                                           const unsigned *__restrict__ list,
                                           const int *__restrict__ origin,
                                           const float4 *__restrict__ node, float4 *acc,
                                           double *accS, unsigned *mumax, const RungArgs &ra,
                                           DevStatus *st, ForceStage *stage,
                                           SinkStage *sstage, int wib, int lane, int A)
{
    const Inst &I = insts[binst[A]];
    const PBox bx = make_pbox(I);
    const Visc vp = {I.alpha, I.beta, I.eps_av, I.qx, I.qx2};
    const int i0 = bstart[A];
    const int i = i0 + lane;
    const int cnt = bucket_len(bstart, A);
    if (cnt == 0) return;  // padding slot
    const bool valid = lane < cnt;
    SinkState s;
    SinkStage &Q = sstage[wib];
    float hs;
    {
        float4 q = valid ? fpos[i] : make_float4(0.f, 0.f, 0.f, 1.f);
        float4 v = valid ? fvel[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 t = valid ? fth[i] : make_float4(0.f, 0.f, 1.f, 1.f);
        hs = q.w;
        s.px = q.x; s.py = q.y; s.pz = q.z;
        s.h2 = q.w * q.w;
        const float ih = 1.f / q.w;
        const float ih2 = ih * ih;
        Q.vel[lane] = v;
        Q.th[lane] = make_float4(t.x, t.y, t.z, q.w);
        Q.ih[lane] = make_float2(ih, K::sigma * ih2 * ih2 * ih);
        s.rg = RUNG && valid ? (int)ra.rung[i] : 0;
        s.rmx = -1;
        s.du = 0.f;
        s.mumax = 0.f;
        s.ax = s.ay = s.az = 0.f;
        s.pairs = 0;
        s.av = 0;
    }
    // sink bounds in the sink frame: cell bound (bc, br), box of balls
    // (gc, gr) and ball of balls (centre gc, radius^2 gR2); wrap decision
    SinkBounds sb;
    bool wrap = false;
    const size_t root = (size_t)I.nbase + 1;
    const float Hmax = node[4 * root + 3].w;  // largest h of the instance (root)
    const float Emax = node[4 * root + 1].w;  // largest bucket extent (root)
    {
        const float p[3] = {s.px, s.py, s.pz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float lo = warp_min(valid ? p[a] : INFINITY), hi = warp_max(valid ? p[a] : -INFINITY);
            float glo = warp_min(valid ? p[a] - hs : INFINITY);
            float ghi = warp_max(valid ? p[a] + hs : -INFINITY);
            sb.bc[a] = 0.5f * (lo + hi);
            sb.br[a] = 0.5f * (hi - lo);
            sb.gc[a] = 0.5f * (glo + ghi);
            sb.gr[a] = 0.5f * (ghi - glo);
            sb.cen[a] = sb.bc[a];
            if (bx.per[a] && (hi - lo) + Hmax + Emax > 0.49f * bx.L[a]) wrap = true;
        }
    }
    {
        float dx = s.px - sb.gc[0], dy = s.py - sb.gc[1], dz = s.pz - sb.gc[2];
        float rr = valid ? sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) + hs : 0.f;
        rr = warp_max(rr) * (1.f + 1e-6f) + I.eps_abs;
        sb.gR2 = rr * rr;
    }
    // fixed point while every bucket-relative coordinate and every pair
    // separation fits 2^31 qx (largest bucket extent and largest h below the
    // limit) and no pair needs its own periodic wrap
    const bool fix = !wrap && Emax < I.fix_lim && Hmax < I.fix_lim;
    if (fix)
        Q.ipos[lane] = valid ? ipos[i] : make_int4(0, 0, 0, 0);
    else
        Q.pos[lane] = make_float4(s.px, s.py, s.pz, 0.f);
    __syncwarp();
    unsigned cands = 0;
    if (fix)
        force_bucket<K, false, true, RUNG>(kp, I, bx, vp, A, lane, stage[wib], Q, s, valid, sb, bstart,
                                     fpos, fvel, fth, ipos, list_cnt, list_off, list, origin,
                                     node, acc, accS, mumax, cands, ra);
    else if (wrap)
        force_bucket<K, true, false, RUNG>(kp, I, bx, vp, A, lane, stage[wib], Q, s, valid, sb, bstart,
                                     fpos, fvel, fth, ipos, list_cnt, list_off, list, origin,
                                     node, acc, accS, mumax, cands, ra);
    else
        force_bucket<K, false, false, RUNG>(kp, I, bx, vp, A, lane, stage[wib], Q, s, valid, sb, bstart,
                                      fpos, fvel, fth, ipos, list_cnt, list_off, list, origin,
                                      node, acc, accS, mumax, cands, ra);
    if (valid) {
        red_add_v4(&acc[i], s.ax, s.ay, s.az, s.du);
        red_add_f64(&accS[i], (double)s.S.s - (double)s.S.c);
        if (s.mumax > 0.f) atomicMax(&mumax[i], __float_as_uint(s.mumax));
        if (RUNG && s.rmx >= 0) atomicMax(&ra.rmax[i], s.rmx);
    }
    unsigned long long wp = warp_sum((unsigned long long)s.pairs);
    unsigned long long wav = warp_sum((unsigned long long)s.av);
    if (lane == 0) {
        atomicAdd(&st->force_pairs, wp);
        atomicAdd(&st->force_av_pairs, wav);
        atomicAdd(&st->force_cand, (unsigned long long)cands * 32ull);
    }
}

// every sink bucket, or (QUEUE: FastGas) the buckets of the queued groups,
// grid-stride
template <class K, bool RUNG, bool QUEUE>
__global__ void __launch_bounds__(128, kForceBlocksPerSM) k_forces(KParams kp, const Inst *__restrict__ insts,
                                                const int *__restrict__ bstart,
                                                const int *__restrict__ binst,
                                                const int *__restrict__ gfirst,
                                                const unsigned *__restrict__ group_ids,
                                                const unsigned *__restrict__ group_cnt,
                                                const float4 *__restrict__ fpos,
                                                const float4 *__restrict__ fvel,
                                                const float4 *__restrict__ fth,
                                                const int4 *__restrict__ ipos,
                                                const unsigned *__restrict__ list_cnt,
                                                const unsigned *__restrict__ list_off,
                                                const unsigned *__restrict__ list,
                                                const int *__restrict__ origin,
                                                const float4 *__restrict__ node, float4 *acc,
                                                double *accS, unsigned *mumax, RungArgs ra,
                                                DevStatus *st)
{
    __shared__ ForceStage stage[kWarpsPerBlock];
    __shared__ SinkStage sstage[kWarpsPerBlock];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bi0 = blockIdx.x * kWarpsPerBlock + wib;
    if (!QUEUE) {
        if (bi0 < kp.nb)
            force_sink<K, RUNG>(kp, insts, bstart, binst, fpos, fvel, fth, ipos, list_cnt,
                                list_off, list, origin, node, acc, accS, mumax, ra, st, stage,
                                sstage, wib, lane, bi0);
        return;
    }
    const int nslots = (int)*group_cnt << kGroupLog;
    for (int bi = bi0; bi < nslots; bi += gridDim.x * kWarpsPerBlock) {
        const int fb = gfirst[group_ids[bi >> kGroupLog]];
        const Inst &Ig = insts[binst[fb]];
        const int j = bi & ((1 << kGroupLog) - 1);
        if (j >= min(Ig.G, Ig.boff + Ig.nb - fb)) continue;
        force_sink<K, RUNG>(kp, insts, bstart, binst, fpos, fvel, fth, ipos, list_cnt, list_off,
                            list, origin, node, acc, accS, mumax, ra, st, stage, sstage, wib,
                            lane, fb + j);
    }
}

// ---------------------------------------------------------------------------
// finalize: PdV term, div v, time-step limits, global minimum
// ---------------------------------------------------------------------------
__global__ void k_finalize(KParams kp, int n, const Inst *__restrict__ insts,
                           const unsigned short *__restrict__ pinst, const float4 *__restrict__ acc,
                           const double *__restrict__ accS, const unsigned *__restrict__ mumax,
                           const float4 *__restrict__ fpos, const float4 *__restrict__ fth,
                           float *ax, float *ay, float *az, float *dudt_h, float *dudt_av,
                           float *divv, float *dt_i, unsigned *dtmin,
                           const double4_16a *__restrict__ acc64, RungArgs ra, DevStatus *st)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float dt = INFINITY;
    int k = -1;
    // hierarchical substep: the inactive particles keep their derivatives
    const bool act = i < n && (!ra.rung || rung_active(ra.sub, ra.R, (int)ra.rung[i]));
    if (act) {
        k = pinst[i];
        const Inst &I = insts[k];
        float4 f;
        if (acc64) {  // FP64 form
            const double4_16a d = acc64[i];
            f = make_float4((float)d.x, (float)d.y, (float)d.z, (float)d.w);
        } else {
            f = acc[i];
        }
        const float S = (float)accS[i];
        const float mu = __uint_as_float(mumax[i]);
        const float4 t = fth[i];
        const float h = fpos[i].w;
        ax[i] = f.x;
        ay[i] = f.y;
        az[i] = f.z;
        dudt_h[i] = t.x * S;
        dudt_av[i] = f.w;
        divv[i] = -S / (t.w * t.z);
        const float amag = sqrtf(fmaf(f.x, f.x, fmaf(f.y, f.y, f.z * f.z)));
        const float dta = amag > 0.f ? I.eta_acc * sqrtf(h / amag) : INFINITY;
        const float dtc = I.eta_courant * h / fmaf(1.f + 0.6f * I.alpha, t.y, 0.6f * I.beta * mu);
        dt = fminf(dta, dtc);
        dt_i[i] = dt;
        if (!(isfinite(f.x) && isfinite(f.y) && isfinite(f.z) && isfinite(f.w) && isfinite(S)))
            raise_status(st, ST_NONFINITE, i);
    }
    // minimum per instance: one atomic per warp when the warp lies in one
    // instance (the usual case), else one per particle
    const int k0 = __shfl_sync(kFull, k, 0);
    if (__all_sync(kFull, k == k0 || k < 0)) {
        dt = warp_min(dt);
        if ((threadIdx.x & 31) == 0 && k0 >= 0 && dt < INFINITY)
            atomicMin(&dtmin[k0], __float_as_uint(dt));
    } else if (k >= 0 && dt < INFINITY) {
        atomicMin(&dtmin[k], __float_as_uint(dt));
    }
}

cudaError_t launch_predict(Ctx &c, const sph_particles &p, cudaStream_t s, const RungArgs *ra)
{
    RungArgs r0{};
    const RungArgs rv = ra ? *ra : r0;
    int n = (int)p.n;
    c.launches += 1;
    const int nt = n > c.kp.ninst ? n : c.kp.ninst;
    const int pr = prof_begin(c, s, SPH_PHASE_PREDICT);
    k_predict<<<(nt + 255) / 256, 256, 0, s>>>(c.kp, n, c.inst, c.pinst, p.v[0], p.v[1], p.v[2],
                                              p.u, p.a[0], p.a[1], p.a[2], p.dudt_h, p.dudt_av,
                                              p.h, p.rho, p.omega, c.pm, c.dts, c.fpos, c.fvel,
                                              c.fth, c.ipos, c.acc, c.accS, c.mumax, c.dtmin,
                                              c.kp.fp64 ? c.fveld : nullptr, c.fthd, c.acc64,
                                              p.divv, p.mat, c.kp.ic ? c.ic_pt : nullptr, rv,
                                              c.st);
    prof_end(c, s, pr);
    return cudaGetLastError();
}

cudaError_t launch_forces(Ctx &c, const sph_particles &p, cudaStream_t s, const RungArgs *ra,
                          bool fastgas)
{
    (void)p;
    const int pr = prof_begin(c, s, SPH_PHASE_FORCES);
    if (c.kp.fp64) {
        const cudaError_t e = launch_forces64(c, s);
        prof_end(c, s, pr);
        return e;
    }
    // FastGas: the buckets of the marked groups, one warp slot per bucket
    // slot of every group (the surplus leaves at once)
    const int slots = fastgas ? c.kp.ng << kGroupLog : c.kp.nb;
    int g = (slots + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const unsigned *gids = fastgas ? c.fg_list : nullptr;
    const unsigned *gcnt = fastgas ? &c.st->fg_cnt : nullptr;
    c.launches += 1;
    RungArgs r0{};
    const RungArgs rv = ra ? *ra : r0;
#define SPH_FORCES_LAUNCH(RUNG_, QUEUE_)                                                  \
    k_forces<KT, RUNG_, QUEUE_><<<g, 32 * kWarpsPerBlock, 0, s>>>(                          \
        c.kp, c.inst, c.bstart, c.binst, c.gfirst, gids, gcnt, c.fpos, c.fvel, c.fth, c.ipos, \
        c.list_cnt, c.list_off, c.list, c.origin, c.node, c.acc, c.accS, c.mumax, rv, c.st)
    SPH_KERNEL_DISPATCH(c.kp.kernel, KT,
        if (rv.rung && fastgas) SPH_FORCES_LAUNCH(true, true);
        else if (rv.rung) SPH_FORCES_LAUNCH(true, false);
        else SPH_FORCES_LAUNCH(false, false);
    )
#undef SPH_FORCES_LAUNCH
    prof_end(c, s, pr);
    return cudaGetLastError();
}

cudaError_t launch_finalize(Ctx &c, const sph_particles &p, cudaStream_t s, const RungArgs *ra)
{
    RungArgs r0{};
    const RungArgs rv = ra ? *ra : r0;
    int n = (int)p.n;
    c.launches += 1;
    const int pr = prof_begin(c, s, SPH_PHASE_FINALIZE);
    k_finalize<<<(n + 255) / 256, 256, 0, s>>>(c.kp, n, c.inst, c.pinst, c.acc, c.accS, c.mumax,
                                               c.fpos, c.fth, p.a[0], p.a[1], p.a[2], p.dudt_h,
                                               p.dudt_av, p.divv, p.dt_i, c.dtmin,
                                               c.kp.fp64 ? c.acc64 : nullptr, rv, c.st);
    prof_end(c, s, pr);
    return cudaGetLastError();
}

}  // namespace sph
