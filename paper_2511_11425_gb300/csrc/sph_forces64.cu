// sph_forces64.cu -- the force pass in the FP64 form (the plain form the
// mixed-precision form is measured against).
//
// The same equations as sph_forces.cu (Sec. 2.3.5 momentum, PdV and
// Monaghan viscosity with the averaged kernel gradient, Eq. AV_heating;
// Sec. 2.3.6 time-step limits), each unordered pair once, with every pair
// term, every sum and both sides' accumulators in FP64:
//   positions   FP64 offsets from the sink bucket's origin (pmd, exact origin
//               offsets), velocities v_pred, A = P/(Omega rho^2) and c from
//               the predictor in FP64
//   sink side   FP64 registers
//   far side    red.global.add.f64 into FP64 accumulators (a xyz, du/dt|Pi, S)
// The candidate culling, the interaction lists and the hit masks are the
// FP32 machinery of the mixed form with radii inflated by 1e-5 h (plus the
// absolute rounding allowance), so they select a superset of the pairs; the
// support test r < max(h_i, h_j) is then taken in FP64 on each hit.
// One warp per sink bucket, two warps per block (the FP64 stage is 14.5 KB
// per warp).
#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int kWarps64 = 2;
constexpr float kInflate = 1e-5f;

struct Sink64 {
    double px, py, pz, h, ih, ih5;
    double vx, vy, vz, m;
    double A, c, rho;
    double ax, ay, az, S, du;
    float mumax;
    float fx, fy, fz, fh2;  // FP32 sink-frame position and inflated h^2 (masks)
    int i;
    unsigned pairs, av;
};

struct Stage64 {
    float4 pos[kChunk];        // FP32 sink-frame position, inflated h^2 (masks)
    double4_16a posd[kChunk];  // FP64 sink-frame position, h
    double4_16a vel[kChunk];   // v_pred, m
    double4_16a th[kChunk];    // A, c, rho, 1/h
    int idx[kChunk];
};

struct Visc64 {
    double alpha, beta, eps_av;
};

template <class K, bool WRAP, bool SELF>
__device__ __forceinline__ void chunk64(const Inst &I, const PBox &bx, const Visc64 &vp,
                                        Stage64 &S, int c, Sink64 &s, bool valid, int lane,
                                        double4_16a *acc64, double *accS, unsigned *mumax)
{
    (void)lane;
    const int nwords = (c + 31) >> 5;
    for (int k = c + lane; k < 32 * nwords; k += 32) {
        S.pos[k] = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
        S.idx[k] = -1;
    }
    __syncwarp();
    unsigned w[4] = {0u, 0u, 0u, 0u};
    if (valid) {
#pragma unroll 1
        for (int ww = 0; ww < nwords; ++ww) {
            unsigned mw = 0u;
#pragma unroll
            for (int b = 31; b >= 0; --b) {
                const float4 q = S.pos[32 * ww + b];
                float dx = s.fx - q.x, dy = s.fy - q.y, dz = s.fz - q.z;
                if (WRAP) {
                    if (bx.per[0]) dx = wrapf(dx, bx.L[0], bx.invL[0]);
                    if (bx.per[1]) dy = wrapf(dy, bx.L[1], bx.invL[1]);
                    if (bx.per[2]) dz = wrapf(dz, bx.L[2], bx.invL[2]);
                }
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                unsigned hit = __float_as_uint(r2 - fmaxf(s.fh2, q.w)) >> 31;
                if (SELF) hit &= S.idx[32 * ww + b] > s.i ? 1u : 0u;
                mw = mw * 2u + hit;
            }
            w[ww] = mw;
        }
    }
    unsigned long long m0 = (unsigned long long)w[0] | ((unsigned long long)w[1] << 32);
    unsigned long long m1 = (unsigned long long)w[2] | ((unsigned long long)w[3] << 32);
    const double sigma = K::sigmad;
    while (m0 | m1) {
        int k;
        if (m0) {
            k = __ffsll((long long)m0) - 1;
            m0 &= m0 - 1ull;
        } else {
            k = 63 + __ffsll((long long)m1);
            m1 &= m1 - 1ull;
        }
        const double4_16a q = S.posd[k];
        double d[3] = {s.px - q.x, s.py - q.y, s.pz - q.z};
        if (WRAP) {
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (bx.per[a]) d[a] -= I.Ld[a] * rint(d[a] * I.invLd[a]);
        }
        const double r2 = fma(d[0], d[0], fma(d[1], d[1], d[2] * d[2]));
        const double hj = q.w;
        if (!(r2 < fmax(s.h * s.h, hj * hj))) continue;  // exact support test
        const double4_16a vj = S.vel[k], tj = S.th[k];
        const double r = sqrt(r2);
        const double ihj = tj.w, qi = r * s.ih, qj = r * ihj;
        const double ihj2 = ihj * ihj;
        const double Fi = qi < 1.0 ? s.ih5 * K::dwqd(qi) : 0.0;
        const double Fj = qj < 1.0 ? sigma * ihj2 * ihj2 * ihj * K::dwqd(qj) : 0.0;
        const double wx = s.vx - vj.x, wy = s.vy - vj.y, wz = s.vz - vj.z;
        const double vr = fma(wx, d[0], fma(wy, d[1], wz * d[2]));
        const bool app = vr < 0.0;
        double Pi = 0.0, mneg = 0.0;
        if (app) {
            const double hb = 0.5 * (s.h + hj), cb = 0.5 * (s.c + tj.y),
                         rb = 0.5 * (s.rho + tj.z);
            const double mu = hb * vr / fma(vp.eps_av * hb, hb, r2);
            Pi = fma(-vp.alpha * cb, mu, vp.beta * mu * mu) / rb;
            mneg = -mu;
        }
        const double Fb = 0.5 * (Fi + Fj);
        const double coef = fma(s.A, Fi, fma(tj.x, Fj, Pi * Fb));
        const double du = 0.5 * Pi * vr * Fb;
        const double cm = coef * vj.w, cs = coef * s.m;
        s.ax = fma(-cm, d[0], s.ax);
        s.ay = fma(-cm, d[1], s.ay);
        s.az = fma(-cm, d[2], s.az);
        s.S = fma(vj.w * vr, Fi, s.S);
        s.du = fma(vj.w, du, s.du);
        const int jj = S.idx[k];
        red_add_f64(&acc64[jj].x, cs * d[0]);
        red_add_f64(&acc64[jj].y, cs * d[1]);
        red_add_f64(&acc64[jj].z, cs * d[2]);
        red_add_f64(&accS[jj], s.m * vr * Fj);
        if (app) {
            red_add_f64(&acc64[jj].w, s.m * du);
            s.mumax = fmaxf(s.mumax, (float)mneg);
            atomicMax(&mumax[jj], __float_as_uint((float)mneg));
            ++s.av;
        }
        ++s.pairs;
    }
    __syncwarp();
}

template <class K, bool WRAP>
__device__ __forceinline__ void bucket64(
    const KParams &kp, const Inst &I, const PBox &bx, const Visc64 &vp, int A, int lane,
    Stage64 &S, Sink64 &s, bool valid, const float *sbc, const float *sbr, const float *sgc,
    const float *sgr, float sgR2, const float *cen, const int *__restrict__ bstart,
    const float4 *__restrict__ fpos, const double4_16a *__restrict__ pmd,
    const double4_16a *__restrict__ fveld, const double4_16a *__restrict__ fthd,
    const unsigned *__restrict__ list_cnt, const unsigned *__restrict__ list_off,
    const unsigned *__restrict__ list, const int *__restrict__ origin,
    const float4 *__restrict__ node, double4_16a *acc64, double *accS, unsigned *mumax,
    unsigned long long &cands)
{
    const unsigned lt = (1u << lane) - 1u;
    const int g = group_of(I, A);
    const unsigned nl = list_cnt[g];
    const unsigned *__restrict__ gl = list + list_off[g];
    // the same list filter as the mixed form (source bucket B >= A whose cell
    // bound meets the sink box-of-balls, or whose box-of-balls meets the sink
    // cell bound; Sec. 2.3.2)
    auto filter_word = [&](unsigned w) -> unsigned {
        const size_t ka = leaf_of(I, A);
        const float4 sb0 = node[4 * ka], sb1 = node[4 * ka + 1];
        const float4 so0 = node[4 * ka + 2], so1 = node[4 * ka + 3];
        const unsigned e = 32 * w + lane;
        bool ok = false;
        if (e < nl) {
            const unsigned B = gl[e];
            const size_t k = leaf_of(I, (int)B);
            if ((int)B >= A) {
                const float4 b0 = node[4 * k], b1 = node[4 * k + 1];
                ok = ovl(so0.x, so1.x, b0.x, b1.x, bx.per[0], bx.L[0], bx.invL[0]) &&
                     ovl(so0.y, so1.y, b0.y, b1.y, bx.per[1], bx.L[1], bx.invL[1]) &&
                     ovl(so0.z, so1.z, b0.z, b1.z, bx.per[2], bx.L[2], bx.invL[2]);
                if (!ok) {
                    const float4 o0 = node[4 * k + 2], o1 = node[4 * k + 3];
                    ok = ovl(sb0.x, sb1.x, o0.x, o1.x, bx.per[0], bx.L[0], bx.invL[0]) &&
                         ovl(sb0.y, sb1.y, o0.y, o1.y, bx.per[1], bx.L[1], bx.invL[1]) &&
                         ovl(sb0.z, sb1.z, o0.z, o1.z, bx.per[2], bx.L[2], bx.invL[2]);
                }
            }
        }
        return __ballot_sync(kFull, ok);
    };
    unsigned myword = 0u;
    for (unsigned w = 0; 32 * w < nl && w < 32; ++w) {
        const unsigned bal = filter_word(w);
        if (lane == (int)w) myword = bal;
    }
    auto stage = [&](int B, int c) -> int {
        float offf[3];
        double offd[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int dk = origin[a * kp.nb + B] - origin[a * kp.nb + A];
            float f = (float)dk * I.qf;
            double fd = (double)dk * I.q;
            if (bx.per[a]) {
                const float nimg = rintf(f * bx.invL[a]);
                f -= bx.L[a] * nimg;
                fd -= I.Ld[a] * (double)nimg;
            }
            offf[a] = f;
            offd[a] = fd;
        }
        const int j = bstart[B] + lane;
        const bool vj = lane < bucket_len(bstart, B);
        const float4 q = vj ? fpos[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float hjc = q.w * (1.f + kInflate) + I.eps_abs;  // culling radius
        float sp[3] = {offf[0] + q.x, offf[1] + q.y, offf[2] + q.z};
        float nw[3] = {0.f, 0.f, 0.f};
        bool gbox = true;
        float dg2 = 0.f, dd = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float dg = sp[a] - sgc[a];
            float dc = sp[a] - sbc[a];
            if (WRAP && bx.per[a]) {
                nw[a] = rintf((sp[a] - cen[a]) * bx.invL[a]);
                sp[a] -= bx.L[a] * nw[a];
                dg = wrapf(dg, bx.L[a], bx.invL[a]);
                dc = wrapf(dc, bx.L[a], bx.invL[a]);
            }
            gbox = gbox && fabsf(dg) <= sgr[a];
            dg2 = fmaf(dg, dg, dg2);
            const float o = fmaxf(fabsf(dc) - sbr[a], 0.f);
            dd = fmaf(o, o, dd);
        }
        const bool in = vj && ((gbox && dg2 <= sgR2) || dd < hjc * hjc);
        const unsigned bal = __ballot_sync(kFull, in);
        if (in) {
            const int pos = c + __popc(bal & lt);
            const double4_16a pd = pmd[j], t = fthd[j];
            S.pos[pos] = make_float4(sp[0], sp[1], sp[2], hjc * hjc);
            S.posd[pos] = make_double4_16a(offd[0] - I.Ld[0] * (double)nw[0] + pd.x,
                                           offd[1] - I.Ld[1] * (double)nw[1] + pd.y,
                                           offd[2] - I.Ld[2] * (double)nw[2] + pd.z,
                                           (double)q.w);
            S.vel[pos] = fveld[j];
            S.th[pos] = make_double4_16a(t.x, t.y, t.z, 1.0 / (double)q.w);
            S.idx[pos] = j;
        }
        return c + __popc(bal);
    };
    int c = stage(A, 0);
    if (c > 0) {
        __syncwarp();
        cands += c;
        chunk64<K, WRAP, true>(I, bx, vp, S, c, s, valid, lane, acc64, accS, mumax);
        c = 0;
    }
    const unsigned nwords = (nl + 31) / 32;
    for (unsigned w = 0; w < nwords; ++w) {
        unsigned mw = w < 32 ? __shfl_sync(kFull, myword, w) : filter_word(w);
        while (mw) {
            const unsigned e = 32 * w + __ffs(mw) - 1;
            mw &= mw - 1u;
            const int B = (int)gl[e];
            if (B == A) continue;
            c = stage(B, c);
            if (c > kChunk - 32) {
                __syncwarp();
                cands += c;
                chunk64<K, WRAP, false>(I, bx, vp, S, c, s, valid, lane, acc64, accS, mumax);
                c = 0;
            }
        }
    }
    if (c > 0) {
        __syncwarp();
        cands += c;
        chunk64<K, WRAP, false>(I, bx, vp, S, c, s, valid, lane, acc64, accS, mumax);
    }
}

template <class K>
__global__ void __launch_bounds__(32 * kWarps64) k_forces64(
    KParams kp, const Inst *__restrict__ insts, const int *__restrict__ bstart,
    const int *__restrict__ binst, const float4 *__restrict__ fpos,
    const double4_16a *__restrict__ pmd, const double4_16a *__restrict__ fveld,
    const double4_16a *__restrict__ fthd, const unsigned *__restrict__ list_cnt,
    const unsigned *__restrict__ list_off, const unsigned *__restrict__ list,
    const int *__restrict__ origin, const float4 *__restrict__ node, double4_16a *acc64,
    double *accS, unsigned *mumax, DevStatus *st)
{
    __shared__ Stage64 stage[kWarps64];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int A = blockIdx.x * kWarps64 + wib;
    if (A >= kp.nb) return;
    const Inst &I = insts[binst[A]];
    const PBox bx = make_pbox(I);
    const Visc64 vp = {(double)I.alpha, (double)I.beta, (double)I.eps_av};
    const int i = bstart[A] + lane;
    const int cnt = bucket_len(bstart, A);
    if (cnt == 0) return;
    const bool valid = lane < cnt;
    Sink64 s;
    {
        const float4 qf = valid ? fpos[i] : make_float4(0.f, 0.f, 0.f, 1.f);
        const double4_16a pd = valid ? pmd[i] : make_double4_16a(0.0, 0.0, 0.0, 0.0);
        const double4_16a v = valid ? fveld[i] : make_double4_16a(0.0, 0.0, 0.0, 0.0);
        const double4_16a t = valid ? fthd[i] : make_double4_16a(0.0, 0.0, 1.0, 1.0);
        s.px = pd.x; s.py = pd.y; s.pz = pd.z;
        s.h = (double)qf.w;
        s.ih = 1.0 / s.h;
        const double ih2 = s.ih * s.ih;
        s.ih5 = K::sigmad * ih2 * ih2 * s.ih;
        s.vx = v.x; s.vy = v.y; s.vz = v.z; s.m = v.w;
        s.A = t.x; s.c = t.y; s.rho = t.z;
        s.ax = s.ay = s.az = s.S = s.du = 0.0;
        s.mumax = 0.f;
        s.fx = qf.x; s.fy = qf.y; s.fz = qf.z;
        const float hc = qf.w * (1.f + kInflate) + I.eps_abs;
        s.fh2 = hc * hc;
        s.i = valid ? i : 0x7fffffff;
        s.pairs = 0;
        s.av = 0;
    }
    // sink bounds in the sink frame with the inflated radius
    float sbc[3], sbr[3], sgc[3], sgr[3], cen[3];
    bool wrap = false;
    const size_t root = (size_t)I.nbase + 1;
    const float Hmax = node[4 * root + 3].w, Emax = node[4 * root + 1].w;
    const float hc = sqrtf(s.fh2);
    {
        const float p[3] = {s.fx, s.fy, s.fz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float lo = warp_min(valid ? p[a] : INFINITY),
                        hi = warp_max(valid ? p[a] : -INFINITY);
            const float glo = warp_min(valid ? p[a] - hc : INFINITY);
            const float ghi = warp_max(valid ? p[a] + hc : -INFINITY);
            sbc[a] = 0.5f * (lo + hi);
            sbr[a] = 0.5f * (hi - lo);
            sgc[a] = 0.5f * (glo + ghi);
            sgr[a] = 0.5f * (ghi - glo);
            cen[a] = sbc[a];
            if (bx.per[a] && (hi - lo) + Hmax + Emax > 0.49f * bx.L[a]) wrap = true;
        }
    }
    float sgR2;
    {
        const float dx = s.fx - sgc[0], dy = s.fy - sgc[1], dz = s.fz - sgc[2];
        float rr = valid ? sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) + hc : 0.f;
        rr = warp_max(rr) * (1.f + 1e-6f) + I.eps_abs;
        sgR2 = rr * rr;
    }
    unsigned long long cands = 0;
    if (wrap)
        bucket64<K, true>(kp, I, bx, vp, A, lane, stage[wib], s, valid, sbc, sbr, sgc, sgr, sgR2,
                          cen, bstart, fpos, pmd, fveld, fthd, list_cnt, list_off, list, origin,
                          node, acc64, accS, mumax, cands);
    else
        bucket64<K, false>(kp, I, bx, vp, A, lane, stage[wib], s, valid, sbc, sbr, sgc, sgr,
                           sgR2, cen, bstart, fpos, pmd, fveld, fthd, list_cnt, list_off, list,
                           origin, node, acc64, accS, mumax, cands);
    if (valid) {
        red_add_f64(&acc64[i].x, s.ax);
        red_add_f64(&acc64[i].y, s.ay);
        red_add_f64(&acc64[i].z, s.az);
        red_add_f64(&acc64[i].w, s.du);
        red_add_f64(&accS[i], s.S);
        if (s.mumax > 0.f) atomicMax(&mumax[i], __float_as_uint(s.mumax));
    }
    const unsigned long long wp = warp_sum((unsigned long long)s.pairs);
    const unsigned long long wav = warp_sum((unsigned long long)s.av);
    if (lane == 0) {
        atomicAdd(&st->force_pairs, wp);
        atomicAdd(&st->force_av_pairs, wav);
        atomicAdd(&st->force_cand, cands * 32ull);
    }
}

}  // namespace

cudaError_t launch_forces64(Ctx &c, cudaStream_t s)
{
    const int g = (c.kp.nb + kWarps64 - 1) / kWarps64;
    c.launches += 1;
    SPH_KERNEL_DISPATCH(c.kp.kernel, KT,
        k_forces64<KT><<<g, 32 * kWarps64, 0, s>>>(c.kp, c.inst, c.bstart, c.binst, c.fpos,
                                                    c.pmd, c.fveld, c.fthd, c.list_cnt,
                                                    c.list_off, c.list, c.origin, c.node,
                                                    c.acc64, c.accS, c.mumax, c.st);
    )
    return cudaGetLastError();
}

}  // namespace sph
