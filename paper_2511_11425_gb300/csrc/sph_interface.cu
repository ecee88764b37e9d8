// sph_interface.cu -- interface correction pass (Sec. 2.3.4).
//
// After the density pass (which left exp(-I_i^2) of the kernel imbalance,
// Eq. Kernel_imbalance, in ic_e) and the predictor (which left P_i and
// T_i = (gamma-1) u_pred,i / R_i in ic_pt), every particle takes the kernel
// averages weighted by exp(-I_j^2) over its neighbours (i itself included),
//     Tbar_i = sum_j T_j e_j W_ij(h_i) / sum_j e_j W_ij(h_i),  Pbar_i likewise,
// the corrected values P~ = e_i P_i + (1 - e_i) Pbar_i, T~ likewise, and the
// corrected density from its material's ideal-gas EOS, rho~ = P~ / (R_i T~).
// The force records then carry rho~: the force pass evaluates the EOS at rho~
// and u_pred, P = (gamma-1) rho~ u_pred = rho~ R_i T_i (the sound speed, a
// function of T alone, is unchanged) and A = P / (Omega rho~^2).
//
// GPU mapping: as the density pass, one warp per sink bucket over its
// group's density list (still in place: the force walk comes after this
// pass), source buckets culled against the warp's box of balls and staged
// 128 at a time in shared memory, per-lane hit masks, evaluation on hits.
// The 1/h^3 and the kernel's normalisation cancel in the averages, so the
// sums use w(q) alone.
#include "sph_internal.cuh"

namespace sph {

namespace {

struct IcStage {
    float4 pos[kChunk];  // source position in the sink frame, e_j
    float2 val[kChunk];  // e_j P_j, e_j T_j
};

template <class K, bool WRAP>
__device__ __forceinline__ void ic_bucket(const KParams &kp, const Inst &I, const PBox &bx, int A,
                                          int lane, IcStage &S, const int *__restrict__ bstart,
                                          const float4 *__restrict__ pm,
                                          const unsigned *__restrict__ list_cnt,
                                          const unsigned *__restrict__ list_off,
                                          const unsigned *__restrict__ list,
                                          const int *__restrict__ origin,
                                          const float4 *__restrict__ node,
                                          const float *__restrict__ h, const float *__restrict__ ic_e,
                                          const float2 *__restrict__ ic_pt, float4 me, bool valid,
                                          const float *cen, float &s_e, float &s_p, float &s_t)
{
    const unsigned lt = (1u << lane) - 1u;
    const int i = bstart[A] + lane;
    const float hi = valid ? h[i] : 0.f;
    const float h2 = hi * hi, ih = valid ? 1.f / hi : 0.f;
    const float p[3] = {me.x, me.y, me.z};
    // the sinks' box of balls in the sink frame, and its absolute centre for
    // the list filter (cell bounds of the source buckets)
    float bc[3], br[3], cc[3], cr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = warp_min(valid ? p[a] - hi : INFINITY);
        const float up = warp_max(valid ? p[a] + hi : -INFINITY);
        bc[a] = 0.5f * (lo + up);
        br[a] = 0.5f * (up - lo) + I.eps_abs;
        cr[a] = br[a] + I.eps_abs;
    }
    {
        float cca = 0.f;
        if (lane < 3) {
            const double o = (double)origin[lane * kp.nb + A] * I.q;
            cca = (float)(o + (double)(lane == 0 ? bc[0] : (lane == 1 ? bc[1] : bc[2])));
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) cc[a] = __shfl_sync(kFull, cca, a);
    }
    const int g = group_of(I, A);
    const unsigned nl = list_cnt[g];
    const unsigned *__restrict__ gl = list + list_off[g];
    float se = 0.f, sp = 0.f, st = 0.f;
    int c = 0;
    auto flush = [&]() {
        const int nwords = (c + 31) >> 5;
        for (int k = c + lane; k < 32 * nwords; k += 32)
            S.pos[k] = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
        __syncwarp();
        if (valid) {
            for (int k = 0; k < 32 * nwords; ++k) {
                const float4 q = S.pos[k];
                float dx = p[0] - q.x, dy = p[1] - q.y, dz = p[2] - q.z;
                if (WRAP) {
                    if (bx.per[0]) dx = wrapf(dx, bx.L[0], bx.invL[0]);
                    if (bx.per[1]) dy = wrapf(dy, bx.L[1], bx.invL[1]);
                    if (bx.per[2]) dz = wrapf(dz, bx.L[2], bx.invL[2]);
                }
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (r2 < h2) {
                    const float w = K::w(r2 * rsqrtf(fmaxf(r2, 1e-37f)) * ih);
                    const float2 v = S.val[k];
                    se = fmaf(q.w, w, se);
                    sp = fmaf(v.x, w, sp);
                    st = fmaf(v.y, w, st);
                }
            }
        }
        __syncwarp();
        c = 0;
    };
    for (unsigned base = 0; base < nl; base += 32) {
        const unsigned e = base + lane;
        bool ok = false;
        if (e < nl) {
            const size_t k = leaf_of(I, (int)gl[e]);
            const float4 b0 = node[4 * k], b1 = node[4 * k + 1];
            ok = ovl(cc[0], cr[0], b0.x, b1.x, bx.per[0], bx.L[0], bx.invL[0]) &&
                 ovl(cc[1], cr[1], b0.y, b1.y, bx.per[1], bx.L[1], bx.invL[1]) &&
                 ovl(cc[2], cr[2], b0.z, b1.z, bx.per[2], bx.L[2], bx.invL[2]);
        }
        unsigned mw = __ballot_sync(kFull, ok);
        while (mw) {
            const int B = (int)gl[base + __ffs(mw) - 1];
            mw &= mw - 1u;
            const float3 off = origin_offset(I, kp.nb, origin, A, B);
            const int j = bstart[B] + lane;
            const bool vj = lane < bucket_len(bstart, B);
            const float4 s = vj ? pm[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            float sp3[3] = {off.x + s.x, off.y + s.y, off.z + s.z};
            bool in = vj;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float d = sp3[a] - bc[a];
                if (WRAP && bx.per[a]) {
                    sp3[a] -= bx.L[a] * rintf((sp3[a] - cen[a]) * bx.invL[a]);
                    d = wrapf(d, bx.L[a], bx.invL[a]);
                }
                in = in && fabsf(d) <= br[a];
            }
            const unsigned bal = __ballot_sync(kFull, in);
            if (in) {
                const int pos = c + __popc(bal & lt);
                const float ej = ic_e[j];
                const float2 pt = ic_pt[j];
                S.pos[pos] = make_float4(sp3[0], sp3[1], sp3[2], ej);
                S.val[pos] = make_float2(ej * pt.x, ej * pt.y);
            }
            c += __popc(bal);
            if (c > kChunk - 32) {
                __syncwarp();
                flush();
            }
        }
    }
    if (c > 0) {
        __syncwarp();
        flush();
    }
    s_e = se;
    s_p = sp;
    s_t = st;
}

template <class K>
__global__ void __launch_bounds__(128) k_interface(
    KParams kp, const Inst *__restrict__ insts, const int *__restrict__ bstart,
    const int *__restrict__ binst, const float4 *__restrict__ pm,
    const unsigned *__restrict__ list_cnt, const unsigned *__restrict__ list_off,
    const unsigned *__restrict__ list, const int *__restrict__ origin,
    const float4 *__restrict__ node, const float *__restrict__ h, const float *__restrict__ ic_e,
    const float2 *__restrict__ ic_pt, const uint8_t *__restrict__ mat, float4 *fth,
    DevStatus *st)
{
    __shared__ IcStage stage[kWarpsPerBlock];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int A = blockIdx.x * kWarpsPerBlock + wib;
    if (A >= kp.nb) return;
    const Inst &I = insts[binst[A]];
    const PBox bx = make_pbox(I);
    const int i = bstart[A] + lane;
    const int cnt = bucket_len(bstart, A);
    if (cnt == 0) return;
    const bool valid = lane < cnt;
    const float4 me = valid ? pm[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    float cen[3];
    bool wrap = false;
    {
        const float hv = valid ? h[i] : 0.f;
        const float Rm = warp_max(hv) + node[4 * ((size_t)I.nbase + 1) + 1].w;
        const float p[3] = {me.x, me.y, me.z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float mn = warp_min(valid ? p[a] : INFINITY);
            const float mx = warp_max(valid ? p[a] : -INFINITY);
            cen[a] = 0.5f * (mn + mx);
            if (bx.per[a] && (mx - mn) + Rm > 0.49f * bx.L[a]) wrap = true;
        }
    }
    float se, sp, stt;
    if (wrap)
        ic_bucket<K, true>(kp, I, bx, A, lane, stage[wib], bstart, pm, list_cnt, list_off, list,
                           origin, node, h, ic_e, ic_pt, me, valid, cen, se, sp, stt);
    else
        ic_bucket<K, false>(kp, I, bx, A, lane, stage[wib], bstart, pm, list_cnt, list_off, list,
                            origin, node, h, ic_e, ic_pt, me, valid, cen, se, sp, stt);
    if (!valid) return;
    const float ei = ic_e[i];
    const float2 pt = ic_pt[i];
    const float pbar = sp / se, tbar = stt / se;
    const float Pc = fmaf(ei, pt.x - pbar, pbar);   // e P + (1 - e) Pbar
    const float Tc = fmaf(ei, pt.y - tbar, tbar);
    const float R = I.r_gas[mat[i] & 3];
    const float rc = Pc / (R * Tc);                  // rho~ from the EOS
    // the force records at rho~: P = rho~ R T (u_pred unchanged), A = P/(Omega rho~^2)
    float4 t = fth[i];
    const float P = rc * R * pt.y;
    t.x = P / (t.w * rc * rc);
    t.z = rc;
    if (!(isfinite(rc) && rc > 0.f && isfinite(t.x))) raise_status(st, ST_NONFINITE, i);
    fth[i] = t;
}

}  // namespace

cudaError_t launch_interface(Ctx &c, const sph_particles &p, cudaStream_t s)
{
    if (c.kp.nb <= 0) return cudaSuccess;
    const int g = (c.kp.nb + kWarpsPerBlock - 1) / kWarpsPerBlock;
    c.launches += 1;
    SPH_KERNEL_DISPATCH(c.kp.kernel, KT,
        k_interface<KT><<<g, 32 * kWarpsPerBlock, 0, s>>>(c.kp, c.inst, c.bstart, c.binst, c.pm,
                                                           c.list_cnt, c.list_off, c.list,
                                                           c.origin, c.node, p.h, c.ic_e,
                                                           c.ic_pt, p.mat, c.fth, c.st);
    )
    return cudaGetLastError();
}

}  // namespace sph
