// sph_fastgas.cu -- FastGas marking for hierarchical steps (Sec. 2.3.6).
//
// On a substep only the particles of the active rungs need new derivatives.
// Their force sums need the densities of their partners: every particle
// that would appear on the interaction list of an active particle.  Those
// are marked, and the density and force passes of the substep then run over
// the marked groups alone (a group is the unit of a list walk, 2^G buckets).
//
// Marking uses the substep's density lists (gathered with radius
// h (1 + margin) round each group's sinks): a group is marked when it holds
// an active particle, or when one of its listed source buckets does (the
// active particle lies within h_j (1 + margin) of a particle j of the group:
// j's scatter partner), and every group whose bucket is listed by a group
// with an active particle is marked too (within h_i (1 + margin) of an
// active i: its gather partner).  A force pair needs r < max(h_i, h_j), so
// each partner of an active particle is marked.  The pairs between two
// unmarked particles, and the densities of unmarked particles, are left as
// they were; the finalize pass writes derivatives of active particles only.
#include "sph_internal.cuh"

namespace sph {

namespace {

// per bucket: does it hold a particle of an active rung (one warp each)
__global__ void k_bucket_active(KParams kp, const int *__restrict__ bstart,
                                const uint8_t *__restrict__ rung, int sub, int R, uint8_t *bact,
                                unsigned *gmark)
{
    const int A = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (A < kp.ng && lane == 0) gmark[A] = 0u;
    if (A >= kp.nb) return;
    const int i = bstart[A] + lane;
    const bool act = lane < bucket_len(bstart, A) && rung_active(sub, R, (int)rung[i]);
    const unsigned any = __ballot_sync(kFull, act);
    if (lane == 0) bact[A] = any ? 1 : 0;
}

// per group (one warp): mark it when it or a listed source bucket holds an
// active particle; when it does, mark the groups of its listed buckets
__global__ void k_mark_groups(KParams kp, const Inst *__restrict__ insts,
                              const int *__restrict__ gfirst, const int *__restrict__ binst,
                              const unsigned *__restrict__ list_cnt,
                              const unsigned *__restrict__ list_off,
                              const unsigned *__restrict__ list, const uint8_t *__restrict__ bact,
                              unsigned *gmark)
{
    const int g = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= kp.ng) return;
    const int fb = gfirst[g];
    const Inst &I = insts[binst[fb]];
    const int nbk = min(I.G, I.boff + I.nb - fb);
    const bool own = __any_sync(kFull, lane < nbk && bact[fb + lane] != 0);
    const unsigned nl = list_cnt[g];
    const unsigned *__restrict__ gl = list + list_off[g];
    bool src = false;
    for (unsigned e = lane; e < nl; e += 32) {
        const int B = (int)gl[e];
        src = src || bact[B] != 0;
        if (own) gmark[group_of(insts[binst[B]], B)] = 1u;
    }
    const bool any_src = __any_sync(kFull, src);
    if (lane == 0 && (own || any_src)) gmark[g] = 1u;
}

// the marked groups into the queue (any order: every group is independent)
__global__ void k_queue_groups(int ng, const unsigned *__restrict__ gmark, unsigned *fg_list,
                               DevStatus *st)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < ng && gmark[g]) fg_list[atomicAdd(&st->fg_cnt, 1u)] = (unsigned)g;
}

}  // namespace

cudaError_t launch_fastgas_mark(Ctx &c, const RungArgs &ra, cudaStream_t s)
{
    const KParams &kp = c.kp;
    if (kp.nb <= 0) return cudaSuccess;
    const int nw = kp.nb > kp.ng ? kp.nb : kp.ng;
    c.launches += 3;
    cudaMemsetAsync(&c.st->fg_cnt, 0, sizeof(unsigned), s);
    k_bucket_active<<<(nw + kWarpsPerBlock - 1) / kWarpsPerBlock, 32 * kWarpsPerBlock, 0, s>>>(
        kp, c.bstart, ra.rung, ra.sub, ra.R, c.bact, c.gmark);
    k_mark_groups<<<(kp.ng + kWarpsPerBlock - 1) / kWarpsPerBlock, 32 * kWarpsPerBlock, 0, s>>>(
        kp, c.inst, c.gfirst, c.binst, c.list_cnt, c.list_off, c.list, c.bact, c.gmark);
    k_queue_groups<<<(kp.ng + 255) / 256, 256, 0, s>>>(kp.ng, c.gmark, c.fg_list, c.st);
    return cudaGetLastError();
}

}  // namespace sph
