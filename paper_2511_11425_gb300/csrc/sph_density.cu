// sph_density.cu -- smoothing length and density (Sec. 2.3.3).
//
// rho_i = sum_j m_j W_ij(h_i) (Eq. Density_estimate), self included, and
// h_i from Newton-Raphson on the constant kernel mass
//     g(h) = 4/3 pi h^3 rho_i(h) / m_i - N_ngb = 4/3 pi sigma S_w / m_i - N_ngb,
//     g'(h) = -4/3 pi sigma S_q / (m_i h),
// with S_w = sum_j m_j w(q_j), S_q = sum_j m_j q_j w'(q_j), q_j = r_ij/h (the h^3
// of W cancels against the h^3 of the kernel volume).  At the converged h
//     rho = sigma S_w / h^3,    Omega = 1 + h/(3 rho) drho/dh = -S_q / (3 S_w).
// The interaction list of each sink bucket was gathered once with radius
// h_seed (1 + margin) (Sec. 2.3.3: the list is kept across iterations and
// over-selects with a slightly larger kernel).  If a particle's h must grow
// past that radius its bucket is queued for a new walk.
//
// GPU mapping: one warp per sink bucket (lane = sink particle).  For each
// Newton pass the warp streams the list: every source bucket is loaded
// coalesced (float4 relative position + mass), moved into the sink frame by
// the exact origin offset, culled against the warp's box of balls and
// compacted into a 128-entry shared-memory chunk.  Each lane then tests all
// chunk entries against its own h (a 128-bit hit mask in registers) and
// evaluates the kernel only on its hits, so the expensive arithmetic runs on
// full warps.  Chunk partial sums are folded into Kahan-compensated totals.
#include <type_traits>

#include "sph_internal.cuh"

namespace sph {


template <bool WRAP>
__device__ __forceinline__ float sep2(const PBox &bx, float px, float py, float pz, float4 q)
{
    float dx = px - q.x, dy = py - q.y, dz = pz - q.z;
    if (WRAP) {
        if (bx.per[0]) dx = wrapf(dx, bx.L[0], bx.invL[0]);
        if (bx.per[1]) dy = wrapf(dy, bx.L[1], bx.invL[1]);
        if (bx.per[2]) dz = wrapf(dz, bx.L[2], bx.invL[2]);
    }
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// Hit masks of one lane against the staged chunk: bit k of word w is set when
// candidate 32w + k lies inside radius^2 (the sign bit of r^2 - h^2, shifted
// in from the top candidate down).  The chunk is padded with NaN positions
// (positive quiet NaN: never a hit) to a multiple of 32, so the fully
// unrolled inner loop needs no bounds checks.
template <bool WRAP>
__device__ __forceinline__ void hit_masks(const PBox &bx, const float4 *cand, int nwords,
                                          float px, float py, float pz, float h2, bool active,
                                          unsigned long long &m0, unsigned long long &m1)
{
    unsigned w0 = 0u, w1 = 0u, w2 = 0u, w3 = 0u;
    if (active) {
#pragma unroll 1
        for (int ww = 0; ww < nwords; ++ww) {
            unsigned mw = 0u;
#pragma unroll
            for (int b = 31; b >= 0; --b) {  // bit b <- sign of r^2 - h^2
                float r2 = sep2<WRAP>(bx, px, py, pz, cand[32 * ww + b]);
                mw = mw * 2u + (__float_as_uint(r2 - h2) >> 31);
            }
            if (ww == 0) w0 = mw; else if (ww == 1) w1 = mw; else if (ww == 2) w2 = mw; else w3 = mw;
        }
    }
    m0 = (unsigned long long)w0 | ((unsigned long long)w1 << 32);
    m1 = (unsigned long long)w2 | ((unsigned long long)w3 << 32);
}

// lowest set bit of m0 | m1 << 64, cleared; without a branch (lanes differ
// in which half is empty)
__device__ __forceinline__ int next_hit(unsigned long long &m0, unsigned long long &m1)
{
    const bool lo = m0 != 0ull;
    const unsigned long long w = lo ? m0 : m1;
    const int k = __ffsll((long long)w) - 1 + (lo ? 0 : 64);
    const unsigned long long w2 = w & (w - 1ull);
    m0 = lo ? w2 : m0;
    m1 = lo ? m1 : w2;
    return k;
}

// the FP64 form's per-lane density sums of one pass
struct DSums {
    double w = 0.0, q = 0.0, qq = 0.0;
};

// per-lane record of the hits with q in [1 - tau, 1 + tau) (shared memory):
// the neighbour count at the Newton-updated h (density_bucket)
constexpr int kShell = 4;

// the interface correction's kernel-imbalance sum (Eq. Kernel_imbalance):
// sum_j kappa_ij (r_j - r_i) m_j w(q_j), kappa = +1 same material, -1 not
struct ImbSum {
    float x = 0.f, y = 0.f, z = 0.f;
};

template <class K, bool WRAP, bool EMIT, bool D64, bool IC>
__device__ __forceinline__ void density_chunk(const PBox &bx, const Inst &I, float4 *cand,
                                              const double4_16a *candd, const int *candj,
                                              const unsigned char *candm, int mat_i, ImbSum &V,
                                              int c, int lane, float px, float py, float pz,
                                              float h2, float ih, const double *pd, double hd,
                                              double ihd, bool active, Kahan &Sw, Kahan &Sq,
                                              Kahan &Sqq, DSums &D, int &cnt, int i,
                                              long long cap, int &emitted, int64_t *ids_out,
                                              const int64_t *__restrict__ id_in, float tau,
                                              float h2e, float *shell, int &ns)
{
    // RELAX: the masks reach h (1 + tau); hits beyond h only enter the shell
    constexpr bool RELAX = !IC && !EMIT;
    const int nwords = (c + 31) >> 5;
    for (int k = c + lane; k < 32 * nwords; k += 32)
        cand[k] = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
    __syncwarp();
    // FP64 form: h2 is the culling radius (inflated over the FP32 rounding
    // of the staged positions); the support test on each hit is exact
    unsigned long long m0, m1;
    hit_masks<WRAP>(bx, cand, nwords, px, py, pz, h2, active, m0, m1);
    int nh = 0;
    if (!D64) {
        float sw = 0.f, sq = 0.f, sqq = 0.f;
        while (m0 | m1) {
            const int k = next_hit(m0, m1);
            const float4 q = cand[k];
            const float r2 = sep2<WRAP>(bx, px, py, pz, q);
            const float r = r2 * rsqrtf(fmaxf(r2, 1e-37f));
            const float qq = r * ih;
            if (RELAX) {
                // inside: the support test the masks make without the shell;
                // shell entries keep q with the sign of that decision
                const bool inside = r2 < h2e;
                if (qq >= 1.f - tau) {
                    if (ns < kShell) shell[ns] = inside ? qq : -qq;
                    ++ns;
                }
                if (!inside) continue;
            }
            const float wv = K::w(qq), dq = K::dwq(qq);
            sw = fmaf(q.w, wv, sw);
            sq = fmaf(q.w * dq, qq * qq, sq);
            if (RELAX) sqq = fmaf(q.w * K::d2w(qq), qq * qq, sqq);
            ++nh;
            if (IC) {
                float dx = q.x - px, dy = q.y - py, dz = q.z - pz;  // r_j - r_i
                if (WRAP) {
                    if (bx.per[0]) dx = wrapf(dx, bx.L[0], bx.invL[0]);
                    if (bx.per[1]) dy = wrapf(dy, bx.L[1], bx.invL[1]);
                    if (bx.per[2]) dz = wrapf(dz, bx.L[2], bx.invL[2]);
                }
                const float kw = (candm[k] == mat_i ? q.w : -q.w) * wv;
                V.x = fmaf(kw, dx, V.x);
                V.y = fmaf(kw, dy, V.y);
                V.z = fmaf(kw, dz, V.z);
            }
            if (EMIT) {
                int j = candj[k];
                if (j != i) {
                    if (emitted < cap) ids_out[(long long)i * cap + emitted] = id_in[j];
                    ++emitted;
                }
            }
        }
        Sw.add(sw);
        Sq.add(sq);
        if (RELAX) Sqq.add(sqq);
    } else {
        const double h2d = hd * hd;
        const double h2o = RELAX ? h2d * (1.0 + (double)tau) * (1.0 + (double)tau) : h2d;
        double sw = 0.0, sq = 0.0, sqq = 0.0;
        while (m0 | m1) {
            const int k = next_hit(m0, m1);
            const double4_16a q = candd[k];
            double d[3] = {pd[0] - q.x, pd[1] - q.y, pd[2] - q.z};
            if (WRAP) {
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    if (bx.per[a]) d[a] -= I.Ld[a] * rint(d[a] * I.invLd[a]);
            }
            const double r2 = fma(d[0], d[0], fma(d[1], d[1], d[2] * d[2]));
            if (!(r2 < h2o)) continue;
            const double qq = sqrt(r2) * ihd;
            if (RELAX) {
                const bool inside = r2 < h2d;
                if (qq >= 1.0 - (double)tau) {
                    if (ns < kShell) shell[ns] = inside ? (float)qq : -(float)qq;
                    ++ns;
                }
                if (!inside) continue;
            }
            sw = fma(q.w, K::wd(qq), sw);
            sq = fma(q.w * K::dwqd(qq), qq * qq, sq);
            if (RELAX) sqq = fma(q.w * K::d2wd(qq), qq * qq, sqq);
            ++nh;
            if (EMIT) {
                int j = candj[k];
                if (j != i) {
                    if (emitted < cap) ids_out[(long long)i * cap + emitted] = id_in[j];
                    ++emitted;
                }
            }
        }
        D.w += sw;
        D.q += sq;
        D.qq += sqq;
    }
    cnt += nh;
}

// D64: the FP64 form (positions from pmd, sums, Newton iteration and the
// outputs' arithmetic in FP64); otherwise FP32 pairs on cell-relative offsets
template <class K, bool WRAP, bool EMIT, bool D64, bool IC>
__device__ __forceinline__ void density_bucket(
    const KParams &kp, const Inst &I, const PBox &bx, int A, int i0, int lane, float4 *cand,
    double4_16a *candd, int *candj, unsigned char *candm, float *shell,
    const uint8_t *__restrict__ mat, float *ic_e, const float4 *__restrict__ pm,
    const double4_16a *__restrict__ pmd, const int *__restrict__ bstart,
    const unsigned *__restrict__ list_cnt,
    const unsigned *__restrict__ list_off, const unsigned *__restrict__ list,
    const int *__restrict__ origin, const float4 *__restrict__ node, float *h_seed, float *h_out,
    float *rho_out, float *omega_out, uint16_t *nngb_out, uint8_t *iters_out, int fixed_h,
    long long cap, uint32_t *count_out, int64_t *ids_out, const int64_t *__restrict__ id_in,
    unsigned *redo_out, unsigned *redo_cnt_out, unsigned *gflag, DevStatus *st, float4 me,
    bool valid, const float *cen)
{
    using Real = typename std::conditional<D64, double, float>::type;
    // step rule (Newton ends once its step is below sqrt(h_rel_tol) h, the
    // outputs moved to the updated h): off for fixed h, the emitting
    // evaluation and the interface correction
    constexpr bool RELAX = !IC && !EMIT;
    const bool relax = RELAX && fixed_h == 0;
    const float tau = relax ? kp.h_step_tol : 0.f;
    float *myshell = RELAX ? shell + lane * kShell : nullptr;
    const unsigned lt = (1u << lane) - 1u;
    const int i = i0 + lane;
    const Real n_ngb = (Real)I.n_ngb;
    const float eps_abs = I.eps_abs;
    Real h = valid ? (Real)h_seed[i] : (Real)1;
    const float R = (float)h * (1.f + kp.margin);  // radius the list was gathered with
    Real lo = 0, hi = (Real)INFINITY;
    bool done = !valid, relist = false, conv = false;
    int iters = 0;
    Real out_h = h, out_rho = 0, out_om = 0;
    int out_n = 0, emitted = 0;
    unsigned long long pairs = 0, cands = 0;
    const float p[3] = {me.x, me.y, me.z};
    double pd[3] = {0.0, 0.0, 0.0};
    if (D64 && valid) {
        const double4_16a q = pmd[i];
        pd[0] = q.x;
        pd[1] = q.y;
        pd[2] = q.z;
    }
    const Real mi = D64 && valid ? (Real)pmd[i].w : (Real)me.w;
    const int mat_i = IC && valid ? (int)mat[i] : 0;
    float out_e = 1.f;  // interface correction: exp(-I^2) at the recorded h
    // Filter the group's list against this bucket's coverage box of balls
    // (radius R): lane w keeps the acceptance bits of entries 32w .. 32w+31
    // of the first 1024.  Longer lists (overflow arena) get the bits of each
    // later word by a ballot when the pass reaches it.
    const int g = group_of(I, A);
    const unsigned nl = list_cnt[g];
    const unsigned *__restrict__ gl = list + list_off[g];
    auto filter_word = [&](unsigned w, const float *cc, const float *cr) -> unsigned {
        const unsigned e = 32 * w + lane;
        bool acc = false;
        if (e < nl) {
            const size_t k = leaf_of(I, (int)gl[e]);
            const float4 b0 = node[4 * k], b1 = node[4 * k + 1];
            acc = ovl(cc[0], cr[0], b0.x, b1.x, bx.per[0], bx.L[0], bx.invL[0]) &&
                  ovl(cc[1], cr[1], b0.y, b1.y, bx.per[1], bx.L[1], bx.invL[1]) &&
                  ovl(cc[2], cr[2], b0.z, b1.z, bx.per[2], bx.L[2], bx.invL[2]);
        }
        return __ballot_sync(kFull, acc);
    };
    auto coverage = [&](float *cc, float *cr) {
        float lo[3], hi[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = warp_min(valid ? p[a] - R : INFINITY);
            hi[a] = warp_max(valid ? p[a] + R : -INFINITY);
            cr[a] = 0.5f * (hi[a] - lo[a]) + 2.f * eps_abs;
        }
        // absolute centre in FP64 (origin + offset, one rounding): axis a in
        // lane a, so the three axes cost one FP64 instruction sequence
        float cca = 0.f;
        if (lane < 3) {
            const int ax = lane;
            const float la = ax == 0 ? lo[0] : (ax == 1 ? lo[1] : lo[2]);
            const float ha = ax == 0 ? hi[0] : (ax == 1 ? hi[1] : hi[2]);
            const double o = (double)origin[ax * kp.nb + A] * I.q;
            cca = (float)(o + 0.5 * ((double)la + (double)ha));
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) cc[a] = __shfl_sync(kFull, cca, a);
    };
    unsigned myword = 0u;
    {
        float cc[3], cr[3];
        coverage(cc, cr);
        for (unsigned w = 0; 32 * w < nl && w < 32; ++w) {
            const unsigned bal = filter_word(w, cc, cr);
            if (lane == (int)w) myword = bal;
        }
    }
    const unsigned nwords = (nl + 31) / 32;

    for (int pass = 0; pass <= kp.max_newton; ++pass) {
        if (__all_sync(kFull, done)) break;
        // culling radius: h itself, or in the FP64 form h inflated over the
        // FP32 rounding of the staged positions (the support test is exact)
        const float hf = D64 ? (float)h * (1.f + 1e-5f) + eps_abs : (float)h;
        const float h2 = hf * hf, ih = 1.f / hf;
        const double ihd = D64 ? 1.0 / (double)h : 0.0;
        // with the step rule (relax) the masks and the culling reach
        // h (1 + tau): the shell of hits the count at the updated h needs
        const float hc = relax ? hf * (1.f + tau) : hf;
        const float h2m = hc * hc;
        // box of balls and ball of balls of the active lanes (Sec. 2.3.2: a
        // source must overlap both shapes)
        float bc[3], br[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float bl = warp_min(done ? INFINITY : p[a] - hc);
            float bh = warp_max(done ? -INFINITY : p[a] + hc);
            bc[a] = 0.5f * (bl + bh);
            br[a] = 0.5f * (bh - bl);
        }
        float bb2;
        {
            float dx = p[0] - bc[0], dy = p[1] - bc[1], dz = p[2] - bc[2];
            float rr = done ? 0.f : sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) + hc;
            rr = warp_max(rr) * (1.f + 1e-6f) + eps_abs;
            bb2 = rr * rr;
        }
        Kahan Sw, Sq, Sqq;
        int ns = 0;
        DSums D;
        ImbSum V;
        int cnt = 0, c = 0;
        for (unsigned w = 0; w < nwords; ++w) {
          unsigned mw;
          if (w < 32) {
            mw = __shfl_sync(kFull, myword, w);
          } else {  // long list: this word's bits now (the box is recomputed)
            float cc[3], cr[3];
            coverage(cc, cr);
            mw = filter_word(w, cc, cr);
          }
          if (!mw) continue;
          // the records of this word's accepted entries, one per lane, fetched
          // together (one round of dependent loads per word, not per entry):
          // first particle, length, origin minus the sink bucket's
          int mj0 = 0, mlen = 0, mdk[3] = {0, 0, 0};
          if ((mw >> lane) & 1u) {
              const int Bm = (int)gl[32 * w + lane];
              mj0 = bstart[Bm];
              mlen = bucket_len(bstart, Bm);
#pragma unroll
              for (int a = 0; a < 3; ++a) mdk[a] = origin[a * kp.nb + Bm] - origin[a * kp.nb + A];
          }
          while (mw) {
            const int l = __ffs(mw) - 1;
            mw &= mw - 1u;
            const int j0 = __shfl_sync(kFull, mj0, l);
            const int len = __shfl_sync(kFull, mlen, l);
            int dk[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) dk[a] = __shfl_sync(kFull, mdk[a], l);
            // origin offset in the sink frame, nearest periodic image
            float off[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float f = (float)dk[a] * I.qf;
                if (bx.per[a]) f -= bx.L[a] * rintf(f * bx.invL[a]);
                off[a] = f;
            }
            const int j = j0 + lane;
            const bool vj = lane < len;
            float4 s = vj ? pm[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            float sp[3] = {off[0] + s.x, off[1] + s.y, off[2] + s.z};
            float nw[3] = {0.f, 0.f, 0.f};  // periodic images moved by the wrap below
            bool in = vj;
            float dd2 = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float d = sp[a] - bc[a];
                if (WRAP && bx.per[a]) {
                    nw[a] = rintf((sp[a] - cen[a]) * bx.invL[a]);
                    sp[a] -= bx.L[a] * nw[a];
                    d = wrapf(d, bx.L[a], bx.invL[a]);
                }
                in = in && fabsf(d) <= br[a];
                dd2 = fmaf(d, d, dd2);
            }
            in = in && dd2 <= bb2;
            unsigned bal = __ballot_sync(kFull, in);
            if (in) {
                int pos = c + __popc(bal & lt);
                cand[pos] = make_float4(sp[0], sp[1], sp[2], s.w);
                if (EMIT) candj[pos] = j;
                if (IC) candm[pos] = mat[j];
                if (D64) {
                    // the same source in FP64: its offset from its own bucket
                    // origin plus the exact origin offset (the image the FP32
                    // offset chose, then the wrap above)
                    const double4_16a sd = pmd[j];
                    double o[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        double f = (double)dk[a] * I.q;
                        if (bx.per[a]) {
                            const float fi = (float)dk[a] * I.qf;
                            f -= I.Ld[a] * (double)rintf(fi * I.invL[a]);
                        }
                        o[a] = f - I.Ld[a] * (double)nw[a];
                    }
                    candd[pos] = make_double4_16a(o[0] + sd.x, o[1] + sd.y, o[2] + sd.z, sd.w);
                }
            }
            c += __popc(bal);
            if (c > kChunk - 32) {
                __syncwarp();
                if (!done) cands += c;
                density_chunk<K, WRAP, EMIT, D64, IC>(bx, I, cand, candd, candj, candm, mat_i, V,
                                                      c, lane, p[0], p[1], p[2], h2m, ih, pd,
                                                      (double)h, ihd, !done, Sw, Sq, Sqq, D, cnt,
                                                      i, cap, emitted, ids_out, id_in, tau, h2,
                                                      myshell, ns);
                __syncwarp();
                c = 0;
            }
          }
        }
        if (c > 0) {
            __syncwarp();
            if (!done) cands += c;
            density_chunk<K, WRAP, EMIT, D64, IC>(bx, I, cand, candd, candj, candm, mat_i, V, c,
                                                  lane, p[0], p[1], p[2], h2m, ih, pd, (double)h,
                                                  ihd, !done, Sw, Sq, Sqq, D, cnt, i, cap,
                                                  emitted, ids_out, id_in, tau, h2, myshell, ns);
            __syncwarp();
        }
        if (!done) {
            ++iters;
            const Real swv = D64 ? (Real)D.w : (Real)Sw.s, sqv = D64 ? (Real)D.q : (Real)Sq.s;
            const Real sigma = D64 ? (Real)K::sigmad : (Real)K::sigma;
            const Real fpt = (Real)4.18879020478639098;  // 4 pi / 3
            const int nn = cnt - 1;  // the particle itself is always in its own list
            pairs += (unsigned long long)(nn > 0 ? nn : 0);
            bool record = fixed_h != 0;
            Real h_final = h;
            if (!record) {
                Real g = fpt * sigma * swv / mi - n_ngb;
                Real dg = -fpt * sigma * sqv / (mi * h);
                if (g < 0) lo = h; else hi = h;
                Real hn = dg > 0 ? h - g / dg : (Real)NAN;
                const Real dh = hn - h;
                // Newton converges quadratically: the updated h lies
                // |g''/(2 g')| dh^2 from the root, with g''/g' = -(2 S_q +
                // S_qq)/(S_q h) from the same sums.  Step rule: accept once
                // that is below h_rel_tol h and |dh| < sqrt(h_rel_tol) h
                // (the width of the shell of hits; the shell must be whole
                // and hn inside the list's radius).  Without the step rule
                // the step itself must be below h_rel_tol h.
                bool step_ok = false;
                if (relax && isfinite(hn) && fabs(dh) < (Real)tau * h && ns <= kShell && hn > 0 &&
                    hn <= (Real)R) {
                    const Real sqqv = D64 ? (Real)D.qq : (Real)Sqq.s;
                    const Real curv = fabs((2 * sqv + sqqv) / (2 * sqv));  // |g''/(2g')| h
                    step_ok = curv * dh * dh < (Real)kp.h_rel_tol * h * h;
                }
                if ((isfinite(hn) && fabs(dh) < (Real)kp.h_rel_tol * h) || step_ok) {
                    // converged: report the Newton update of the last
                    // evaluation
                    record = true;
                    h_final = hn;
                } else {
                    if (!(hn > lo && hn < hi)) hn = isfinite(hi) ? (Real)0.5 * (lo + hi) : 2 * h;
                    if (hn > (Real)R) {
                        if (h >= (Real)R) {  // g(R) < 0: the root lies beyond the list's coverage
                            relist = true;
                            done = true;
                            out_h = hn;
                        } else {
                            hn = (Real)R;
                        }
                    }
                    if (!done) {
                        if (iters >= kp.max_newton) {
                            done = true;
                            raise_status(st, ST_NOCONV, i);
                        } else {
                            h = hn;
                        }
                    }
                }
            }
            if (record) {
                done = true;
                conv = true;
                out_h = h_final;
                const Real ihr = (Real)1 / h;
                out_rho = sigma * swv * ihr * ihr * ihr;
                out_om = -sqv / (3 * swv);
                if (!D64) {  // the FP32 form keeps its arithmetic as FP32 ops
                    out_rho = (Real)(K::sigma * (float)swv * ih * ih * ih);
                }
                out_n = nn;
                if (relax && h_final != h) {
                    // rho, Omega and n_i at the reported h: the sums moved
                    // to first order in dh (dS_w/dh = -S_q/h and dS_q/dh =
                    // -(S_q + S_qq)/h with S_qq = sum m q^2 w''(q)), the
                    // count from the shell of hits near q = 1
                    const Real dh = h_final - h;
                    const Real sqqv = D64 ? (Real)D.qq : (Real)Sqq.s;
                    const Real swn = swv - dh * sqv / h;
                    const Real sqn = sqv - dh * (sqv + sqqv) / h;
                    const Real ihn = (Real)1 / h_final;
                    out_rho = sigma * swn * ihn * ihn * ihn;
                    out_om = -sqn / (3 * swn);
                    if (ns <= kShell) {
                        const float ratio = (float)(h_final / h);
                        for (int k = 0; k < ns; ++k) {
                            const float v = myshell[k];
                            if (ratio >= 1.f && v < 0.f && -v < ratio) ++out_n;
                            if (ratio < 1.f && v > 0.f && v >= ratio) --out_n;
                        }
                    }
                }
                if (IC) {  // Eq. Kernel_imbalance: I = alpha |V| / (h sum m w)
                    const float vm = sqrtf(fmaf(V.x, V.x, fmaf(V.y, V.y, V.z * V.z)));
                    const float Ii = I.ic_alpha * vm / ((float)h * (float)swv);
                    out_e = __expf(-Ii * Ii);
                }
                if (!(isfinite(out_rho) && isfinite(out_om) && out_rho > 0))
                    raise_status(st, ST_NONFINITE, i);
                if ((float)h >= I.hcap) raise_status(st, ST_ARG, i);
            }
        }
    }
    if (valid && !done) raise_status(st, ST_NOCONV, i);
    bool any_relist = __any_sync(kFull, relist);
    if (any_relist) {
        if (valid) h_seed[i] = (float)(relist ? out_h : (conv ? out_h : h));
        if (lane == 0 && atomicOr(&gflag[g], 1u) == 0u) {
            if (redo_out) {
                unsigned pos = atomicAdd(redo_cnt_out, 1u);
                redo_out[pos] = (unsigned)g;
            } else {
                raise_status(st, ST_NOCONV, i);  // no re-walk round left
            }
        }
    } else if (valid && conv) {
        h_out[i] = (float)out_h;
        rho_out[i] = (float)out_rho;
        omega_out[i] = (float)out_om;
        nngb_out[i] = (uint16_t)min(out_n, 65535);
        iters_out[i] = (uint8_t)min(iters, 255);
        if (EMIT && count_out) count_out[i] = (uint32_t)out_n;
        if (IC) ic_e[i] = out_e;
    }
    unsigned long long wp = warp_sum(pairs), wc = warp_sum(cands);
    int wi = (int)warp_max((float)iters);
    if (lane == 0) {
        atomicAdd(&st->density_pairs, wp);
        atomicAdd(&st->density_cand, wc);
        atomicMax(&st->max_iters, wi);
    }
}

// one sink bucket A (one warp)
template <class K, bool EMIT, bool D64, bool IC>
__device__ __forceinline__ void density_slot(
    const uint8_t *__restrict__ mat, float *ic_e, unsigned char *candm, float *shell,
    const KParams &kp, const Inst *__restrict__ insts, const float4 *__restrict__ pm,
    const double4_16a *__restrict__ pmd, const int *__restrict__ bstart,
    const int *__restrict__ binst, const unsigned *__restrict__ list_cnt,
    const unsigned *__restrict__ list_off, const unsigned *__restrict__ list,
    const int *__restrict__ origin, float *h_seed, float *h_out, float *rho_out,
    float *omega_out, uint16_t *nngb_out, uint8_t *iters_out, int fixed_h, long long cap,
    uint32_t *count_out, int64_t *ids_out, const int64_t *__restrict__ id_in,
    unsigned *redo_out, unsigned *redo_cnt_out, unsigned *gflag,
    const float4 *__restrict__ node, float4 *leaf_out, DevStatus *st, float4 *cand,
    double4_16a *candd, int *candj, int A, int lane)
{
    const Inst &I = insts[binst[A]];
    const PBox bx = make_pbox(I);
    const int i0 = bstart[A];
    const int i = i0 + lane;
    const int cnt = bucket_len(bstart, A);
    if (cnt == 0) return;  // padding slot
    const bool valid = lane < cnt;
    const float4 me = valid ? pm[i] : make_float4(0.f, 0.f, 0.f, 1.f);
    // sink centre (periodic images are chosen nearest to it) and whether
    // pair separations need their own minimum-image wrap
    float cen[3];
    bool wrap = false;
    {
        const float R = valid ? h_seed[i] * (1.f + kp.margin) : 0.f;
        const float Rm = warp_max(R) + node[4 * ((size_t)I.nbase + 1) + 1].w;  // + largest bucket extent
        const float p[3] = {me.x, me.y, me.z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float mn = warp_min(valid ? p[a] : INFINITY), mx = warp_max(valid ? p[a] : -INFINITY);
            cen[a] = 0.5f * (mn + mx);
            if (bx.per[a] && (mx - mn) + Rm > 0.49f * bx.L[a]) wrap = true;
        }
    }
    if (wrap)
        density_bucket<K, true, EMIT, D64, IC>(kp, I, bx, A, i0, lane, cand, candd, candj, candm,
                                               shell, mat, ic_e, pm, pmd,
                                           bstart, list_cnt, list_off, list, origin, node, h_seed,
                                           h_out, rho_out, omega_out, nngb_out, iters_out, fixed_h,
                                           cap, count_out, ids_out, id_in, redo_out, redo_cnt_out,
                                           gflag, st, me, valid, cen);
    else
        density_bucket<K, false, EMIT, D64, IC>(kp, I, bx, A, i0, lane, cand, candd, candj,
                                                candm, shell, mat, ic_e, pm, pmd,
                                            bstart, list_cnt, list_off, list, origin, node, h_seed,
                                            h_out, rho_out, omega_out, nngb_out, iters_out,
                                            fixed_h, cap, count_out, ids_out, id_in, redo_out,
                                            redo_cnt_out, gflag, st, me, valid, cen);
    // the leaf's box of balls with the new h (the bounds update after the
    // density pass, Sec. 2.3.3): positions relative to the bucket origin
    // (pm) widened by h, absolute centre in FP64 (origin + offset, one
    // rounding) with axis a in lane a, half widths inflated by the rounding
    // allowance.  Only the cell bounds of sources are read above, so the
    // box of balls of any leaf may change while other warps run.
    const float hv = valid ? h_out[i] : 0.f;
    const float pr[3] = {me.x, me.y, me.z};
    float mnb[3], mxb[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        mnb[a] = warp_min(valid ? pr[a] - hv : INFINITY);
        mxb[a] = warp_max(valid ? pr[a] + hv : -INFINITY);
    }
    const float hmax = warp_max(hv);
    float oca = 0.f, ora = 0.f;
    if (lane < 3) {
        const int ax = lane;
        const double o = (double)origin[ax * kp.nb + A] * I.q;
        const float mna = ax == 0 ? mnb[0] : (ax == 1 ? mnb[1] : mnb[2]);
        const float mxa = ax == 0 ? mxb[0] : (ax == 1 ? mxb[1] : mxb[2]);
        oca = (float)(o + 0.5 * ((double)mna + (double)mxa));
        ora = 0.5f * (mxa - mna) + I.eps_abs;
    }
    float oc[3], orr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        oc[a] = __shfl_sync(kFull, oca, a);
        orr[a] = __shfl_sync(kFull, ora, a);
    }
    if (lane == 0) {
        const size_t k = (size_t)I.nbase + I.P + (A - I.boff);
        leaf_out[4 * k + 2] = make_float4(oc[0], oc[1], oc[2], 0.f);
        leaf_out[4 * k + 3] = make_float4(orr[0], orr[1], orr[2], hmax);
    }
}

template <class K, bool EMIT, bool D64, bool IC>
// 5 blocks of 4 warps per SM: the register cap (96) measured faster than
// the compiler's own choice (about 128 registers, 4 blocks)
__global__ void __launch_bounds__(128, 5) k_density(
    const uint8_t *__restrict__ mat, float *ic_e, KParams kp, const Inst *__restrict__ insts, const float4 *__restrict__ pm,
    const double4_16a *__restrict__ pmd, const int *__restrict__ bstart,
    const int *__restrict__ binst, const int *__restrict__ gfirst,
    const unsigned *__restrict__ list_cnt, const unsigned *__restrict__ list_off,
    const unsigned *__restrict__ list, const int *__restrict__ origin,
    const unsigned *__restrict__ group_ids, const unsigned *__restrict__ group_cnt,
    float *h_seed, float *h_out, float *rho_out, float *omega_out, uint16_t *nngb_out,
    uint8_t *iters_out, int fixed_h, long long cap, uint32_t *count_out, int64_t *ids_out,
    const int64_t *__restrict__ id_in, unsigned *redo_out, unsigned *redo_cnt_out,
    unsigned *gflag, const float4 *__restrict__ node, float4 *leaf_out, DevStatus *st)
{
    __shared__ float4 cand_s[kWarpsPerBlock][kChunk];
    __shared__ double4_16a candd_s[D64 ? kWarpsPerBlock : 1][D64 ? kChunk : 1];
    __shared__ int candj_s[EMIT ? kWarpsPerBlock : 1][EMIT ? kChunk : 1];
    __shared__ unsigned char candm_s[IC ? kWarpsPerBlock : 1][IC ? kChunk : 1];
    constexpr bool RELAX = !IC && !EMIT;
    __shared__ float shell_s[RELAX ? kWarpsPerBlock : 1][RELAX ? 32 * kShell : 1];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double4_16a *candd = D64 ? candd_s[wib] : nullptr;
    if (!group_ids) {  // every bucket, one warp each
        const int A = blockIdx.x * kWarpsPerBlock + wib;
        if (A < kp.nb)
            density_slot<K, EMIT, D64, IC>(mat, ic_e, IC ? candm_s[wib] : nullptr, RELAX ? shell_s[wib] : nullptr, kp, insts, pm, pmd, bstart, binst, list_cnt, list_off, list,
                                       origin, h_seed, h_out, rho_out, omega_out, nngb_out,
                                       iters_out, fixed_h, cap, count_out, ids_out, id_in,
                                       redo_out, redo_cnt_out, gflag, node, leaf_out, st, cand_s[wib],
                                       candd, EMIT ? candj_s[wib] : nullptr, A, lane);
        return;
    }
    // the buckets of the groups queued for this re-walk round (8 warp slots
    // per queued group), grid-stride: the grid is small and mostly idle
    const int nslots = (int)*group_cnt << kGroupLog;
    for (int bi = blockIdx.x * kWarpsPerBlock + wib; bi < nslots;
         bi += gridDim.x * kWarpsPerBlock) {
        const int fb = gfirst[group_ids[bi >> kGroupLog]];
        const Inst &Ig = insts[binst[fb]];
        const int j = bi & ((1 << kGroupLog) - 1);
        if (j >= min(Ig.G, Ig.boff + Ig.nb - fb)) continue;
        density_slot<K, EMIT, D64, IC>(mat, ic_e, IC ? candm_s[wib] : nullptr, RELAX ? shell_s[wib] : nullptr, kp, insts, pm, pmd, bstart, binst, list_cnt, list_off, list,
                                   origin, h_seed, h_out, rho_out, omega_out, nngb_out, iters_out,
                                   fixed_h, cap, count_out, ids_out, id_in, redo_out, redo_cnt_out,
                                   gflag, node, leaf_out, st, cand_s[wib], candd,
                                   EMIT ? candj_s[wib] : nullptr, fb + j, lane);
    }
}


__global__ void k_isentropic(int n, const Inst *__restrict__ insts,
                             const unsigned short *__restrict__ pinst,
                             const float *__restrict__ rho, const float *__restrict__ rho_old,
                             double *u, const DevStatus *st)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || st->code != 0) return;  // no state change after an error
    float ro = rho_old[i];
    const double g1 = (double)insts[pinst[i]].gamma - 1.0;
    if (ro > 0.f) u[i] *= pow((double)rho[i] / (double)ro, g1);
}

cudaError_t launch_density(Ctx &c, const sph_particles &p, const float *h_seed, int round,
                           int fixed_h, int64_t cap, uint32_t *count, int64_t *ids,
                           cudaStream_t s, bool fastgas)
{
    const KParams &kp = c.kp;
    if (kp.nb <= 0) return cudaSuccess;
    // round < 0: every bucket (FastGas: the buckets of the marked groups),
    // queueing re-walks for round 0; round r: the buckets of the groups
    // queued for round r, queueing for round r + 1.  A re-walk round covers
    // the queued groups with a small grid-stride grid, the FastGas pass with
    // one warp slot per bucket slot of every group (the surplus leaves at once)
    const int slots = round < 0 && !fastgas ? kp.nb : kp.ng << kGroupLog;
    int g = (slots + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (round >= 0 && g > kRoundBlocks) g = kRoundBlocks;
    const bool emit = ids != nullptr || count != nullptr;
    const unsigned *gids = round < 0 ? (fastgas ? c.fg_list : nullptr)
                                     : c.redo + (size_t)round * kp.ng;
    const unsigned *gcnt = round < 0 ? (fastgas ? &c.st->fg_cnt : nullptr)
                                     : &c.st->redo_cnt[round];
    const int next = round + 1;
    unsigned *redo_out = next < kRelistRounds ? c.redo + (size_t)next * kp.ng : nullptr;
    unsigned *redo_cnt_out = next < kRelistRounds ? &c.st->redo_cnt[next] : nullptr;
    cudaMemsetAsync(c.gflag, 0, sizeof(unsigned) * (size_t)kp.ng, s);
    c.launches += 1;
    const int pr = prof_begin(c, s, SPH_PHASE_DENSITY);
    // the evolved density mode keeps p.rho as state: the kernel sum goes to
    // scratch (h and Omega to p as always)
    float *rho_out = kp.evolved ? c.rho_sum : p.rho;
#define SPH_DENSITY_LAUNCH(EMIT_, D64_, IC_)                                                 \
    k_density<KT, EMIT_, D64_, IC_><<<g, 32 * kWarpsPerBlock, 0, s>>>(                            \
        p.mat, c.ic_e, kp, c.inst, c.pm, c.pmd, c.bstart, c.binst, c.gfirst, c.list_cnt, c.list_off, c.list,     \
        c.origin, gids, gcnt, (float *)h_seed, p.h, rho_out, p.omega, p.nngb, p.iters, fixed_h,   \
        (long long)cap, count, ids, p.id, redo_out, redo_cnt_out, c.gflag, c.node, c.node, c.st)
    SPH_KERNEL_DISPATCH(kp.kernel, KT,
        if (kp.fp64) {
            if (emit) SPH_DENSITY_LAUNCH(true, true, false);
            else SPH_DENSITY_LAUNCH(false, true, false);
        } else if (kp.ic && !emit) {
            SPH_DENSITY_LAUNCH(false, false, true);
        } else {
            if (emit) SPH_DENSITY_LAUNCH(true, false, false);
            else SPH_DENSITY_LAUNCH(false, false, false);
        }
    )
#undef SPH_DENSITY_LAUNCH
    prof_end(c, s, pr);
    return cudaGetLastError();
}

cudaError_t launch_isentropic(Ctx &c, const sph_particles &p, cudaStream_t s)
{
    int n = (int)p.n;
    c.launches += 1;
    k_isentropic<<<(n + 255) / 256, 256, 0, s>>>(n, c.inst, c.pinst, p.rho, c.rho_old, p.u,
                                                 c.st);
    return cudaGetLastError();
}

}  // namespace sph
