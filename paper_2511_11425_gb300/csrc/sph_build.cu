// sph_build.cu -- sph_build_cells and the interaction-list walk.
//
// Sec. 2.1 keeps particles ordered so that every tree cell is a contiguous
// range; Sec. 2.3.2 bounds every cell by the box of its particles (cell
// bound) and the box of the particles' kernel balls (box-of-balls), merged
// bottom-up, and finds interaction partners of a whole group at once by
// overlap tests of those bounds.  Here the order is a 30-bit curve order per
// instance (stable LSD radix sort of (instance, curve index) keys, so
// instances keep their particle ranges), a bucket is up to 32 consecutive
// particles of one instance inside one small key cell (one warp), and each
// instance has an implicit complete binary tree over its bucket slots.  Every
// phase is one launch over all instances.
#include "sph_internal.cuh"
#include "sph_bits.h"

namespace sph {

// ---------------------------------------------------------------------------
// bounding boxes of open axes (periodic axes use the box); grid (chunks, ninst)
// ---------------------------------------------------------------------------
__global__ void k_bbox_partial(const Inst *__restrict__ insts, const double *__restrict__ x,
                               const double *__restrict__ y, const double *__restrict__ z,
                               double *part)
{
    const Inst &I = insts[blockIdx.y];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = I.off + blockIdx.x * blockDim.x + threadIdx.x; i < I.off + I.n;
         i += gridDim.x * blockDim.x) {
        double v[3] = {x[i], y[i], z[i]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mn[a] = fmin(mn[a], v[a]);
            mx[a] = fmax(mx[a], v[a]);
        }
    }
    __shared__ double smn[3][32], smx[3][32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double a0 = warp_min(mn[a]), a1 = warp_max(mx[a]);
        if (lane == 0) { smn[a][w] = a0; smx[a][w] = a1; }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        int nw = blockDim.x >> 5;
        double *out = part + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * 6;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double a0 = lane < nw ? smn[a][lane] : INFINITY;
            double a1 = lane < nw ? smx[a][lane] : -INFINITY;
            a0 = warp_min(a0);
            a1 = warp_max(a1);
            if (lane == 0) {
                out[a] = a0;
                out[3 + a] = a1;
            }
        }
    }
}

// key box per instance = [lo0..2, cells per unit length 0..2, cubes0..2, bin]
__global__ void k_bbox_final(KParams kp, const Inst *__restrict__ insts, const double *part,
                             double *morton_box, DevStatus *st)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kp.ninst) return;
    const Inst &I = insts[k];
    // The domain is cut into near-cubes: round(extent / S) per axis, S = the
    // shortest extent (at least 1/1024 of the longest), visited in a snake
    // order (every cube is a face neighbour of the one before); the curve
    // orders the particles inside each cube on 2^bin cells per axis.  Key
    // cells stay near-cubic (aspect below 3/2) however elongated the domain
    // (a tube, a slab), so curve ranges stay compact, and no thin sliver
    // cube is left at the far faces.
    double lo3[3], ext3[3], emin = INFINITY, emax = 0.0;
    for (int a = 0; a < 3; ++a) {
        double lo, hi;
        if (I.periodic[a] || !kp.any_open || I.n == 0) {
            lo = I.lo[a];
            hi = I.hi[a];
        } else {
            lo = INFINITY;
            hi = -INFINITY;
            for (int b = 0; b < kBboxChunks; ++b) {
                lo = fmin(lo, part[((size_t)k * kBboxChunks + b) * 6 + a]);
                hi = fmax(hi, part[((size_t)k * kBboxChunks + b) * 6 + 3 + a]);
            }
        }
        if (!isfinite(lo) || !isfinite(hi)) {
            raise_status(st, ST_NONFINITE, k);
            lo = 0.0;
            hi = 1.0;
        }
        lo3[a] = lo;
        ext3[a] = hi - lo;
        emin = fmin(emin, hi - lo);
        emax = fmax(emax, hi - lo);
    }
    const double S = fmax(emin, emax / (double)(1 << kMortonBits)) + 1e-300;
    long long ncubes = 1;
    int nc[3];
    for (int a = 0; a < 3; ++a) {
        nc[a] = (int)fmin(fmax(rint(ext3[a] / S), 1.0), (double)(1 << kMortonBits));
        ncubes *= nc[a];
    }
    int bpre = 0;
    while ((1ll << bpre) < ncubes) ++bpre;
    const int bin = min(kMortonBits, (30 - bpre) / 3);
    double *mb = morton_box + kKeyBox * k;
    // integers are stored as their bit patterns (readers decode them
    // without FP64 conversions); slot 10 holds the FP32 side of one key cell
    for (int a = 0; a < 3; ++a) {
        mb[a] = lo3[a];
        mb[3 + a] = ldexp((double)nc[a], bin) / (ext3[a] * (1.0 + 1e-9) + 1e-300);
        mb[6 + a] = __longlong_as_double((long long)nc[a]);
    }
    mb[9] = __longlong_as_double((long long)bin);
    const float cell = 1.f / fminf(fminf((float)mb[3], (float)mb[4]), (float)mb[5]);
    mb[10] = __longlong_as_double((long long)__float_as_uint(cell));
}

// 10-bit coordinate -> every third bit of a 30-bit word
__device__ __forceinline__ unsigned spread3(unsigned x)
{
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

// Hilbert index of a 10-bit cell (Skilling 2004, "Programming the Hilbert
// curve"): the axes are turned into the transposed index by undoing, level
// by level from the top, the reflections and axis exchanges of the curve,
// then Gray-decoded; the transposed bits interleaved (axis 0 highest in each
// triple) are the index.  Cells consecutive on the curve share a face.
__device__ __forceinline__ unsigned hilbert3(unsigned c0, unsigned c1, unsigned c2, int bits)
{
    if (bits <= 0) return 0u;
    unsigned X[3] = {c0, c1, c2};
    for (unsigned Q = 1u << (bits - 1); Q > 1u; Q >>= 1) {
        const unsigned P = Q - 1u;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (X[a] & Q) {
                X[0] ^= P;  // reflect the low bits of axis 0
            } else {        // exchange the low bits of axes 0 and a
                const unsigned t = (X[0] ^ X[a]) & P;
                X[0] ^= t;
                X[a] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    unsigned t = 0;
    for (unsigned Q = 1u << (bits - 1); Q > 1u; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1u;
    X[0] ^= t;
    X[1] ^= t;
    X[2] ^= t;
    return (spread3(X[0]) << 2) | (spread3(X[1]) << 1) | spread3(X[2]);
}

// key = instance << 30 | snake index of the cube << 3 bin | curve index in
// the cube (at most 30 bits per instance)
__global__ void k_morton(int n, const Inst *__restrict__ insts,
                         const unsigned short *__restrict__ pinst,
                         const double *__restrict__ x, const double *__restrict__ y,
                         const double *__restrict__ z, const double *__restrict__ mbox,
                         unsigned long long *keys, unsigned int *vals)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = pinst[i];
    const double *mb = mbox + kKeyBox * k;
    const int bin = (int)__double_as_longlong(mb[9]);
    const double v[3] = {x[i], y[i], z[i]};
    unsigned cube[3], w[3], nc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        nc[a] = (unsigned)__double_as_longlong(mb[6 + a]);
        // cell index: truncation toward zero, then clamped to the key box
        // in integers (a NaN converts to 0)
        const long long tl = __double2ll_rz((v[a] - mb[a]) * mb[3 + a]);
        const long long top = ((long long)nc[a] << bin) - 1;
        const unsigned ti = (unsigned)(tl < 0 ? 0 : (tl > top ? top : tl));
        cube[a] = ti >> bin;
        w[a] = ti & ((1u << bin) - 1u);
    }
    // snake: layers along axis 2, rows along axis 1, reversed on odd layers
    // and odd rows, so consecutive cubes share a face
    const unsigned r = cube[2] * nc[1] + ((cube[2] & 1u) ? nc[1] - 1u - cube[1] : cube[1]);
    const unsigned cidx = r * nc[0] + ((r & 1u) ? nc[0] - 1u - cube[0] : cube[0]);
    const unsigned in = insts[k].curve == SPH_CURVE_HILBERT
                            ? hilbert3(w[0], w[1], w[2], bin)
                            : spread3(w[0]) | (spread3(w[1]) << 1) | (spread3(w[2]) << 2);
    keys[i] = ((unsigned long long)k << 30) | ((unsigned long long)cidx << (3 * bin)) | in;
    vals[i] = (unsigned)i;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (instance, curve index) keys, 8-bit digits, tiles of
// 2048 keys (256 threads x 8).  Per pass: tile histograms, a per-digit scan
// over the tiles (one block per digit), and a stable scatter whose ranks
// come from warp-level match_any in key order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_sort_hist(const unsigned long long *__restrict__ keys,
                                                   int n, int shift, unsigned *hist, int ntiles)
{
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * kSortTile;
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        int i = base + k * 256 + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// block d: exclusive scan of digit d's counts over the tiles; total -> tot[d]
__global__ void __launch_bounds__(1024) k_sort_rowscan(unsigned *hist, int ntiles, unsigned *tot)
{
    __shared__ unsigned part[1024];
    unsigned *row = hist + (size_t)blockIdx.x * ntiles;
    int t = threadIdx.x;
    int per = (ntiles + 1023) / 1024;
    int b0 = min(ntiles, t * per), b1 = min(ntiles, b0 + per);
    unsigned s = 0;
    for (int k = b0; k < b1; ++k) s += row[k];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        unsigned v = t >= o ? part[t - o] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    unsigned run = part[t] - s;
    for (int k = b0; k < b1; ++k) {
        unsigned c = row[k];
        row[k] = run;
        run += c;
    }
    if (t == 1023) tot[blockIdx.x] = part[1023];
}

__global__ void __launch_bounds__(256) k_sort_scatter(const unsigned long long *__restrict__ kin,
                                                      const unsigned *__restrict__ vin,
                                                      unsigned long long *__restrict__ kout,
                                                      unsigned *__restrict__ vout, int n,
                                                      int shift, const unsigned *__restrict__ hist,
                                                      const unsigned *__restrict__ tot, int ntiles)
{
    __shared__ unsigned wcnt[8][256];
    __shared__ unsigned toff[256];
    __shared__ unsigned base_s[256];
    int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int k = tid; k < 8 * 256; k += 256) (&wcnt[0][0])[k] = 0;
    base_s[tid] = tot[tid];
    __syncthreads();
    // exclusive prefix of the digit totals (Hillis-Steele in shared memory)
    for (int o = 1; o < 256; o <<= 1) {
        unsigned v = tid >= o ? base_s[tid - o] : 0u;
        __syncthreads();
        base_s[tid] += v;
        __syncthreads();
    }
    toff[tid] = base_s[tid] - tot[tid] + hist[tid * ntiles + blockIdx.x];
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long key[kSortItems];
    unsigned val[kSortItems], rnk[kSortItems];
    const int per_warp = 32 * kSortItems;
    int base = blockIdx.x * kSortTile + w * per_warp;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int i = base + r * 32 + lane;
        bool ok = i < n;
        key[r] = ok ? kin[i] : 0ull;
        val[r] = ok ? vin[i] : 0u;
        unsigned d = ok ? (unsigned)((key[r] >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(kFull, d);
        unsigned before = 0;
        if (ok) before = wcnt[w][d];
        __syncwarp();
        rnk[r] = before + __popc(peers & lt);
        if (ok && lane == __ffs(peers) - 1) wcnt[w][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        unsigned s = 0;
        for (int k = 0; k < 8; ++k) {
            unsigned c = wcnt[k][tid];
            wcnt[k][tid] = s;
            s += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int i = base + r * 32 + lane;
        if (i < n) {
            unsigned d = (unsigned)((key[r] >> shift) & 255u);
            unsigned pos = toff[d] + wcnt[w][d] + rnk[r];
            kout[pos] = key[r];
            vout[pos] = val[r];
        }
    }
}

// ---------------------------------------------------------------------------
// in-place permutation of every caller array through one scratch buffer
// ---------------------------------------------------------------------------
struct PermFields {
    unsigned long long *f8[8];
    float *f4[11];
    uint16_t *f2;
    uint8_t *f1;
    uint8_t *f1b;  // material ids (may be NULL)
};

__global__ void k_gather_all(const unsigned *__restrict__ perm, int n, PermFields pf, char *tmp)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned j = perm[i];
    unsigned long long *t8 = (unsigned long long *)tmp;
    float *t4 = (float *)(t8 + (size_t)8 * n);
    uint16_t *t2 = (uint16_t *)(t4 + (size_t)11 * n);
    uint8_t *t1 = (uint8_t *)(t2 + n);
#pragma unroll
    for (int f = 0; f < 8; ++f) t8[(size_t)f * n + i] = pf.f8[f][j];
#pragma unroll
    for (int f = 0; f < 11; ++f) t4[(size_t)f * n + i] = pf.f4[f][j];
    t2[i] = pf.f2[j];
    t1[i] = pf.f1[j];
    if (pf.f1b) t1[n + i] = pf.f1b[j];
}

__global__ void k_copyback_all(int n, PermFields pf, const char *tmp)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long *t8 = (const unsigned long long *)tmp;
    const float *t4 = (const float *)(t8 + (size_t)8 * n);
    const uint16_t *t2 = (const uint16_t *)(t4 + (size_t)11 * n);
    const uint8_t *t1 = (const uint8_t *)(t2 + n);
#pragma unroll
    for (int f = 0; f < 8; ++f) pf.f8[f][i] = t8[(size_t)f * n + i];
#pragma unroll
    for (int f = 0; f < 11; ++f) pf.f4[f][i] = t4[(size_t)f * n + i];
    pf.f2[i] = t2[i];
    pf.f1[i] = t1[i];
    if (pf.f1b) pf.f1b[i] = t1[n + i];
}

// ---------------------------------------------------------------------------
// bucket layout.  The paper splits cells until a leaf holds few particles
// (Sec. 2.3.2); here the curve-ordered particles are cut into warps that do
// not straddle large octree cells.  Particle i gets a position P(i) in a
// padded index space of its instance (bucket slot = P / 32, group = slot /
// G): P = 0 at the instance's first particle and P(i) = align(P(i-1) + 1,
// a_i), where a_i = 32 G when the smallest key cell holding particles i-1 and
// i is wider than group_cell h (a new group starts), 32 when it is wider than
// bucket_cell h (a new bucket starts), else 1.  The maps
// x -> align(x + c, a) + d with power-of-two a are closed under composition,
// so P is one parallel scan (tile reduce, scan of the tile totals, apply).
// An instance whose layout needs more slots than it has keeps plain
// 32-particle chunks.
// ---------------------------------------------------------------------------
struct PadF {
    int reset, c, a, d;  // x -> align((reset ? -1 : x) + c, a) + d
};

__device__ __forceinline__ int align_up(int v, int a) { return ((v + a - 1) / a) * a; }

// f first, then g
__device__ __forceinline__ PadF pad_then(PadF f, PadF g)
{
    if (g.reset) return g;
    const int e = f.d + g.c;
    if (g.a <= f.a) return PadF{f.reset, f.c, f.a, align_up(e, g.a) + g.d};
    return PadF{f.reset, f.c + f.a * ((e + f.a - 1) / f.a), g.a, g.d};
}

__device__ __forceinline__ int pad_apply(PadF f) { return align_up(f.c - 1, f.a) + f.d; }

__device__ __forceinline__ PadF pad_shfl_up(PadF f, int o)
{
    return PadF{__shfl_up_sync(kFull, f.reset, o), __shfl_up_sync(kFull, f.c, o),
                __shfl_up_sync(kFull, f.a, o), __shfl_up_sync(kFull, f.d, o)};
}

__device__ __forceinline__ PadF pad_elem(int i, const Inst *__restrict__ insts,
                                         const unsigned short *__restrict__ pinst,
                                         const unsigned long long *__restrict__ keys,
                                         const float *__restrict__ h,
                                         const double *__restrict__ mbox)
{
    const int k = pinst[i];
    const Inst &I = insts[k];
    if (i == I.off) return PadF{1, 1, 1, 0};
    const double *mb = mbox + kKeyBox * k;
    const int bin = (int)__double_as_longlong(mb[9]);
    const unsigned long long x = keys[i - 1] ^ keys[i];
    const int d = x ? 63 - __clzll((long long)x) : -1;
    const int ga = kBucket * I.G;
    if (d >= 3 * bin) return PadF{0, 1, ga, 0};  // another cube of the snake
    // the smallest common cell has 2^(d/3 + 1) key cells per side
    const float cell = __uint_as_float((unsigned)__double_as_longlong(mb[10]));
    const float side = ldexpf(cell, d < 0 ? 0 : d / 3 + 1);
    const float hh = fmaxf(h[i - 1], h[i]);
    const int a = side > I.kg * hh ? ga : (side > I.kb * hh ? kBucket : 1);
    return PadF{0, 1, a, 0};
}

// composition of the 8 consecutive items of each thread, then of the block
__global__ void __launch_bounds__(256) k_pad_reduce(int n, const Inst *__restrict__ insts,
                                                    const unsigned short *__restrict__ pinst,
                                                    const unsigned long long *__restrict__ keys,
                                                    const float *__restrict__ h,
                                                    const double *__restrict__ mbox, int4 *agg)
{
    __shared__ PadF wtot[8];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int base = blockIdx.x * kPadTile + t * 8;
    PadF f = {0, 0, 1, 0};
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (base + q < n) f = pad_then(f, pad_elem(base + q, insts, pinst, keys, h, mbox));
    // inclusive scan over the warp (its last lane holds the warp total)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const PadF u = pad_shfl_up(f, o);
        if (lane >= o) f = pad_then(u, f);
    }
    if (lane == 31) wtot[w] = f;
    __syncthreads();
    if (t == 0) {
        PadF tot = wtot[0];
        for (int k = 1; k < 8; ++k) tot = pad_then(tot, wtot[k]);
        agg[blockIdx.x] = make_int4(tot.reset, tot.c, tot.a, tot.d);
    }
}

// exclusive scan of the tile totals, in place (one block)
__global__ void __launch_bounds__(1024) k_pad_scan(int ntiles, int4 *agg)
{
    __shared__ PadF part[1024];
    const int t = threadIdx.x;
    const int per = (ntiles + 1023) / 1024;
    const int b0 = min(ntiles, t * per), b1 = min(ntiles, b0 + per);
    PadF f = {0, 0, 1, 0};
    for (int k = b0; k < b1; ++k) {
        const int4 v = agg[k];
        f = pad_then(f, PadF{v.x, v.y, v.z, v.w});
    }
    part[t] = f;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const PadF u = t >= o ? part[t - o] : PadF{0, 0, 1, 0};
        __syncthreads();
        if (t >= o) part[t] = pad_then(u, part[t]);
        __syncthreads();
    }
    PadF run = t > 0 ? part[t - 1] : PadF{0, 0, 1, 0};
    for (int k = b0; k < b1; ++k) {
        const int4 v = agg[k];
        agg[k] = make_int4(run.reset, run.c, run.a, run.d);
        run = pad_then(run, PadF{v.x, v.y, v.z, v.w});
    }
}

// every slot starts out empty at its instance's end
__global__ void k_pad_init(int nb, const Inst *__restrict__ insts, const int *__restrict__ binst,
                           int *bstart)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const Inst &I = insts[binst[b]];
    bstart[b] = I.off + I.n;
}

// positions P(i); a particle that starts a bucket writes its slot and the
// padding slots before it; the last particle of an instance reports the
// slots used
__global__ void __launch_bounds__(256) k_pad_apply(int n, const Inst *__restrict__ insts,
                                                   const unsigned short *__restrict__ pinst,
                                                   const unsigned long long *__restrict__ keys,
                                                   const float *__restrict__ h,
                                                   const double *__restrict__ mbox,
                                                   const int4 *__restrict__ excl, int *bstart,
                                                   int *used)
{
    __shared__ PadF wtot[8];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int base = blockIdx.x * kPadTile + t * 8;
    PadF f = {0, 0, 1, 0};
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (base + q < n) f = pad_then(f, pad_elem(base + q, insts, pinst, keys, h, mbox));
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const PadF u = pad_shfl_up(f, o);
        if (lane >= o) f = pad_then(u, f);
    }
    if (lane == 31) wtot[w] = f;
    PadF lane_ex = pad_shfl_up(f, 1);
    if (lane == 0) lane_ex = PadF{0, 0, 1, 0};
    __syncthreads();
    const int4 ev = excl[blockIdx.x];
    PadF run = PadF{ev.x, ev.y, ev.z, ev.w};
    for (int k = 0; k < w; ++k) run = pad_then(run, wtot[k]);
    run = pad_then(run, lane_ex);
    int prev = pad_apply(run);  // P of the item before this thread's first
    for (int q = 0; q < 8; ++q) {
        const int i = base + q;
        if (i >= n) break;
        const PadF e = pad_elem(i, insts, pinst, keys, h, mbox);
        run = pad_then(run, e);
        const int P = pad_apply(run);
        const int k = pinst[i];
        const Inst &I = insts[k];
        const int slot = P >> 5;
        if ((P & 31) == 0) {
            const int s0 = e.reset ? slot : (prev >> 5) + 1;
            for (int sl = s0; sl <= slot && sl < I.nb; ++sl) bstart[I.boff + sl] = i;
        }
        if (i == I.off + I.n - 1) used[k] = slot + 1;
        prev = P;
    }
}

// instances whose layout did not fit keep plain 32-particle chunks
__global__ void k_pad_fallback(int nb, const Inst *__restrict__ insts,
                               const int *__restrict__ binst, const int *__restrict__ used,
                               int *bstart)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int k = binst[b];
    const Inst &I = insts[k];
    if (used[k] <= I.nb) return;
    bstart[b] = min(I.off + kBucket * (b - I.boff), I.off + I.n);
}

// ---------------------------------------------------------------------------
// buckets: origin, relative positions, leaf bounds.  One warp per bucket.
// Offsets from the bucket's first particle are formed in FP64 (minimum image
// on periodic axes) and every reduction runs in FP32 on those offsets.
// update_pos = 1: a re-sort (new origins); 2: a refit without a re-sort
// (the origins are kept).  The box of balls from the h of the density pass
// (Sec. 2.3.3) is written by the density kernel for each bucket it solves.
// ---------------------------------------------------------------------------

// round to nearest even of v inv as an int, for inv a power of two and
// |v inv| < 2^31: v inv is exact, and adding 1.5 2^52 in the same FMA rounds
// it to an integer held in the low word (one FP64 instruction instead of a
// multiply and a conversion; the result equals __double2int_rn(v * inv))
__device__ __forceinline__ int fix_rn(double v, double inv)
{
    return __double2loint(fma(v, inv, 6755399441055744.0));
}
__global__ void __launch_bounds__(128) k_buckets(KParams kp, const Inst *__restrict__ insts,
                                                 const int *__restrict__ bstart,
                                                 const int *__restrict__ binst,
                                                 const double *__restrict__ x,
                                                 const double *__restrict__ y,
                                                 const double *__restrict__ z,
                                                 const float *__restrict__ m,
                                                 const float *__restrict__ h, int *origin,
                                                 float4 *pm, int4 *ipos, double4_16a *pmd,
                                                 float4 *node, int update_pos, DevStatus *st)
{
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= kp.nb) return;
    const Inst &I = insts[binst[b]];
    const int i0 = bstart[b];
    const int i = i0 + lane;
    const int cnt = bucket_len(bstart, b);
    if (cnt == 0) {  // padding slot: an empty leaf
        if (lane == 0) {
            const size_t k = (size_t)I.nbase + I.P + (b - I.boff);
            const float4 e = make_float4(0.f, 0.f, 0.f, 0.f), er = make_float4(-1.f, -1.f, -1.f, 0.f);
            for (int a = 0; a < 3; ++a) origin[a * kp.nb + b] = 0;
            node[4 * k + 0] = e;
            node[4 * k + 1] = er;
            node[4 * k + 2] = e;
            node[4 * k + 3] = er;
        }
        return;
    }
    // FP64 runs at a small fraction of the FP32 rate on this part, and an
    // FP64 instruction costs the pipe about as much for one active lane as
    // for 32: each lane does only its own offset in FP64 (one subtract and
    // one fused rounding to fixed point per axis; the minimum-image wrap
    // only when the offset could exceed half a period), the warp-uniform
    // origin and bounds arithmetic runs one axis per lane, all axes in one
    // instruction, and the conversions between the formats run on the
    // integer pipes (sph_bits.h, the same values as the hardware's).
    const bool ok = lane < cnt;
    const int ax = lane < 3 ? lane : 0;  // the axis of lanes 0, 1, 2
    auto sel = [&](const auto *v3) { return ax == 0 ? v3[0] : (ax == 1 ? v3[1] : v3[2]); };
    const double inv_qx = bits::f2d(I.inv_qx);  // a power of two
    float rel[3];
    double o3 = 0.0;  // lanes 0, 1, 2: origin of axis `ax` (grid index times q, exact)
    if (update_pos == 2) {
        // refit (no re-sort): the bucket keeps its origin grid point, and each
        // lane's offset from it is one FP64 subtraction per axis (nearest
        // periodic image of the origin)
        double v[3] = {0.0, 0.0, 0.0};
        if (ok) { v[0] = x[i]; v[1] = y[i]; v[2] = z[i]; }
        if (lane < 3) o3 = bits::i2d_pow2(origin[ax * kp.nb + b], I.q);
        int fix[3];
        double rdd[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double rd = v[a] - __shfl_sync(kFull, o3, a);
            float rf = bits::d2f(rd);
            if (I.periodic[a] && fabsf(rf) > 0.49f * I.L[a]) {
                rd -= I.Ld[a] * rint(rd * I.invLd[a]);
                rf = bits::d2f(rd);
            }
            rdd[a] = rd;
            rel[a] = rf;
            fix[a] = fix_rn(rd, inv_qx);
        }
        if (ok) {
            if (!(isfinite(rel[0]) && isfinite(rel[1]) && isfinite(rel[2])))
                raise_status(st, ST_NONFINITE, i);
            pm[i] = make_float4(rel[0], rel[1], rel[2], m[i]);
            ipos[i] = make_int4(fix[0], fix[1], fix[2], 0);
            if (pmd) pmd[i] = make_double4_16a(rdd[0], rdd[1], rdd[2], (double)m[i]);
        }
    } else {
        double v[3] = {0.0, 0.0, 0.0};
        if (ok) { v[0] = x[i]; v[1] = y[i]; v[2] = z[i]; }
        double first[3], d[3];
        float mnd[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            first[a] = __shfl_sync(kFull, v[a], 0);
            d[a] = v[a] - first[a];
            float df = bits::d2f(d[a]);
            if (I.periodic[a] && fabsf(df) > 0.49f * I.L[a]) {
                d[a] -= I.Ld[a] * rint(d[a] * I.invLd[a]);
                df = bits::d2f(d[a]);
            }
            mnd[a] = warp_min(ok ? df : INFINITY);
        }
        double fo = 0.0;  // first - origin of axis `ax` (lanes 0, 1, 2)
        if (lane < 3) {
            const double fa = sel(first);
            double kd = floor((fa + bits::f2d(sel(mnd))) * I.inv_q);
            if (!(fabs(kd) < 1073741824.0)) {  // the grid index must fit an int
                raise_status(st, ST_ARG, b);
                kd = 0.0;
            }
            origin[ax * kp.nb + b] = (int)kd;
            o3 = kd * I.q;
            fo = fa - o3;
        }
        int fix[3];
        double rdd[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double rd = __shfl_sync(kFull, fo, a) + d[a];
            rdd[a] = rd;
            rel[a] = bits::d2f(rd);
            // fixed point in units of qx (garbage if the bucket is wider than
            // the fixed-point range; the force kernel then does not use it)
            fix[a] = fix_rn(rd, inv_qx);
        }
        if (ok) {
            if (!(isfinite(rel[0]) && isfinite(rel[1]) && isfinite(rel[2])))
                raise_status(st, ST_NONFINITE, i);
            pm[i] = make_float4(rel[0], rel[1], rel[2], m[i]);
            ipos[i] = make_int4(fix[0], fix[1], fix[2], 0);
            if (pmd) pmd[i] = make_double4_16a(rdd[0], rdd[1], rdd[2], (double)m[i]);
        }
    }
    const float hi = ok ? h[i] : 0.f;
    if (ok && !(hi > 0.f && isfinite(hi))) raise_status(st, ST_NONFINITE, i);
    float mn[3], mx[3], mnb[3], mxb[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        mn[a] = warp_min(ok ? rel[a] : INFINITY);
        mx[a] = warp_max(ok ? rel[a] : -INFINITY);
        mnb[a] = warp_min(ok ? rel[a] - hi : INFINITY);
        mxb[a] = warp_max(ok ? rel[a] + hi : -INFINITY);
    }
    const float hmax = warp_max(hi);
    // absolute centres (FP64 add of the origin, then one rounding) and half
    // widths inflated by the rounding allowance: the bucket box of axis a in
    // lane a, the box of balls of axis a in lane 3 + a
    const int a6 = lane < 3 ? lane : (lane < 6 ? lane - 3 : 0);
    const double o6 = __shfl_sync(kFull, o3, a6);
    float cen = 0.f, hw = 0.f;
    if (lane < 6) {
        auto sel6 = [&](const float *v3) { return a6 == 0 ? v3[0] : (a6 == 1 ? v3[1] : v3[2]); };
        const bool ball = lane >= 3;
        const float lo = ball ? sel6(mnb) : sel6(mn), up = ball ? sel6(mxb) : sel6(mx);
        cen = bits::d2f(o6 + 0.5 * (bits::f2d(lo) + bits::f2d(up)));
        hw = 0.5f * (up - lo) + I.eps_abs;
    }
    float bc[3], br[3], oc[3], orr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        bc[a] = __shfl_sync(kFull, cen, a);
        br[a] = __shfl_sync(kFull, hw, a);
        oc[a] = __shfl_sync(kFull, cen, 3 + a);
        orr[a] = __shfl_sync(kFull, hw, 3 + a);
    }
    if (lane == 0) {
        const size_t k = (size_t)I.nbase + I.P + (b - I.boff);
        // .w of the cell half widths: the bucket's largest full extent
        float ext = 2.f * fmaxf(br[0], fmaxf(br[1], br[2]));
        node[4 * k + 0] = make_float4(bc[0], bc[1], bc[2], 0.f);
        node[4 * k + 1] = make_float4(br[0], br[1], br[2], ext);
        node[4 * k + 2] = make_float4(oc[0], oc[1], oc[2], 0.f);
        node[4 * k + 3] = make_float4(orr[0], orr[1], orr[2], hmax);
    }
}

// union of two centre/half-width intervals; on periodic axes the second is
// first moved to its image nearest the first; r < 0 marks an empty interval
__device__ __forceinline__ void union1(float c1, float r1, float c2, float r2, bool per, float L,
                                       float invL, float eps, float &c, float &r)
{
    if (r1 < 0.f) { c = c2; r = r2; return; }
    if (r2 < 0.f) { c = c1; r = r1; return; }
    if (per) c2 = c1 + wrapf(c2 - c1, L, invL);
    float lo = fminf(c1 - r1, c2 - r2), hi = fmaxf(c1 + r1, c2 + r2);
    c = 0.5f * (lo + hi);
    r = 0.5f * (hi - lo) + eps;
    if (per && r >= 0.5f * L) r = L;  // covers the whole periodic axis
}

__device__ __forceinline__ void union_pair(const Inst &I, const float4 *a, const float4 *b,
                                           float4 *out, int s)
{
    float4 c1 = a[2 * s], r1 = a[2 * s + 1], c2 = b[2 * s], r2 = b[2 * s + 1];
    float cc[3], rr[3];
    float a1[3] = {c1.x, c1.y, c1.z}, b1[3] = {r1.x, r1.y, r1.z};
    float a2[3] = {c2.x, c2.y, c2.z}, b2[3] = {r2.x, r2.y, r2.z};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
        union1(a1[ax], b1[ax], a2[ax], b2[ax], I.periodic[ax], I.L[ax], I.invL[ax], I.eps_abs,
               cc[ax], rr[ax]);
    out[2 * s] = make_float4(cc[0], cc[1], cc[2], 0.f);
    out[2 * s + 1] = make_float4(rr[0], rr[1], rr[2], fmaxf(r1.w, r2.w));
}

// Bottom-up merge of the bounds (Sec. 2.3.2).  Each block follows one entry
// of the refit schedule: it loads 2^levels consecutive nodes of level `lvl`
// of one instance's tree into shared memory and reduces them to one node of
// level lvl - levels.  Leaves of padding buckets are written empty.
__global__ void __launch_bounds__(256) k_tree_levels(const Inst *__restrict__ insts,
                                                     const RefitBlock *__restrict__ sched,
                                                     float4 *node, int bob_only)
{
    __shared__ float4 sn[256][4];
    const RefitBlock rb = sched[blockIdx.x];
    const Inst &I = insts[rb.inst];
    const int width = 1 << rb.levels;
    const int t = threadIdx.x;
    const unsigned first = (1u << rb.lvl) + (unsigned)rb.blk * width;
    if (t < width) {
        const unsigned k = first + t;
        float4 *nd = node + 4 * ((size_t)I.nbase + k);
        if (rb.lvl == I.logP && (int)(k - I.P) >= I.nb) {
            float4 e = make_float4(0.f, 0.f, 0.f, 0.f), er = make_float4(-1.f, -1.f, -1.f, 0.f);
            sn[t][0] = e; sn[t][1] = er; sn[t][2] = e; sn[t][3] = er;
            if (!bob_only) { nd[0] = e; nd[1] = er; }
            nd[2] = e;
            nd[3] = er;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) sn[t][q] = nd[q];
        }
    }
    __syncthreads();
    for (int l = 0; l < rb.levels; ++l) {
        const int cnt = width >> (l + 1);
        float4 out[4];
        if (t < cnt) {
            out[0] = sn[2 * t][0];
            out[1] = sn[2 * t][1];
            if (!bob_only) union_pair(I, sn[2 * t], sn[2 * t + 1], out, 0);
            union_pair(I, sn[2 * t], sn[2 * t + 1], out, 1);
        }
        __syncthreads();
        if (t < cnt) {
            const unsigned k = (first >> (l + 1)) + t;
            float4 *nd = node + 4 * ((size_t)I.nbase + k);
            if (!bob_only) {
                sn[t][0] = out[0];
                sn[t][1] = out[1];
                nd[0] = out[0];
                nd[1] = out[1];
            }
            sn[t][2] = out[2];
            sn[t][3] = out[3];
            nd[2] = out[2];
            nd[3] = out[3];
        }
        __syncthreads();
    }
}

static void tree_refit(Ctx &c, cudaStream_t s, int bob_only)
{
    size_t off = 0;
    for (int nblk : c.refit_band) {
        if (nblk > 0) {
            k_tree_levels<<<nblk, 256, 0, s>>>(c.inst, c.refit + off, c.node, bob_only);
            c.launches += 1;
        }
        off += nblk;
    }
}

// ---------------------------------------------------------------------------
// interaction-list walk (Sec. 2.3.2): one walk per GROUP of up to 8
// consecutive buckets (256 particles, the paper's GPU group size) of one
// instance, breadth-first over that instance's tree, one round of node loads per level.
//   density: source cell bound overlaps the group's box of balls of radius
//            h_walk (1 + margin)                              (gather)
//   force:   source cell bound overlaps the group box-of-balls (gather) OR
//            source box-of-balls overlaps the group cell bound (scatter),
//            restricted to source buckets >= the group's first bucket
// The list holds source bucket ids; each sink bucket of the group filters it
// against its own bounds inside the pair kernels.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void walk_group(const KParams &kp, const Inst *__restrict__ insts,
                                           const int *__restrict__ gfirst,
                                           const int *__restrict__ bstart,
                                           const int *__restrict__ binst, int mode,
                                           const float4 *__restrict__ node,
                                           const float4 *__restrict__ pm,
                                           const int *__restrict__ origin,
                                           const float *__restrict__ h_walk, unsigned *list,
                                           unsigned *list_cnt, unsigned *list_off,
                                           unsigned *arena_used, unsigned arena_cap,
                                           DevStatus *st, unsigned (*buf)[kWalkCap], int g,
                                           int lane)
{
    const int fb = gfirst[g];
    const Inst &I = insts[binst[fb]];
    const int nbg = min(I.G, I.boff + I.nb - fb);
    const int fl = fb - I.boff;  // local index of the group's first bucket
    if (bstart[fb + nbg] == bstart[fb]) {  // only padding slots
        if (lane == 0) {
            list_cnt[g] = 0u;
            list_off[g] = (unsigned)g * kWalkCap;
        }
        return;
    }

    // group bounds in absolute (unwrapped) f32 coordinates
    float gc[3], gr[3], sc[3], sr[3];  // gather box, group cell box
    if (mode == WALK_DENSITY) {
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        // unrolled over the group's (at most 8) buckets so that their loads
        // are issued together
#pragma unroll
        for (int j = 0; j < (1 << kGroupLog); ++j) {
            if (j >= nbg) break;
            const int b = fb + j;
            const float3 off = origin_offset(I, kp.nb, origin, fb, b);
            const int i0 = bstart[b];
            if (lane < bucket_len(bstart, b)) {
                const int i = i0 + lane;
                const float4 r = pm[i];
                const float R = h_walk[i] * (1.f + kp.margin);
                const float p[3] = {off.x + r.x, off.y + r.y, off.z + r.z};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    lo[a] = fminf(lo[a], p[a] - R);
                    hi[a] = fmaxf(hi[a], p[a] + R);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = warp_min(lo[a]);
            hi[a] = warp_max(hi[a]);
            gr[a] = 0.5f * (hi[a] - lo[a]) + 2.f * I.eps_abs;
            sr[a] = -1.f;
        }
        // absolute centre in FP64 (origin + offset, one rounding), axis a in
        // lane a: one FP64 instruction sequence for the three axes
        float gca = 0.f;
        if (lane < 3) {
            const int ax = lane;
            const float la = ax == 0 ? lo[0] : (ax == 1 ? lo[1] : lo[2]);
            const float ha = ax == 0 ? hi[0] : (ax == 1 ? hi[1] : hi[2]);
            const double o = (double)origin[ax * kp.nb + fb] * I.q;
            gca = (float)(o + 0.5 * ((double)la + (double)ha));
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gc[a] = __shfl_sync(kFull, gca, a);
            sc[a] = gc[a];
        }
    } else {
        const size_t k = (size_t)I.nbase + (I.P >> I.logG) + (fl >> I.logG);
        float4 b0 = node[4 * k], b1 = node[4 * k + 1], o0 = node[4 * k + 2], o1 = node[4 * k + 3];
        gc[0] = o0.x; gc[1] = o0.y; gc[2] = o0.z;
        gr[0] = o1.x; gr[1] = o1.y; gr[2] = o1.z;
        sc[0] = b0.x; sc[1] = b0.y; sc[2] = b0.z;
        sr[0] = b1.x; sr[1] = b1.y; sr[2] = b1.z;
    }

    const float4 *tn = node + 4 * (size_t)I.nbase;  // this instance's tree
    // does node nd (at level lvl), with cell bound (b0, b1) and box of balls
    // (o0, o1; force walks only), hold sources of this group?
    auto accept_b = [&](unsigned nd, int lvl, float4 b0, float4 b1, float4 o0,
                        float4 o1) -> bool {
        if (!(b1.x >= 0.f)) return false;  // empty
        bool gth = ovl(gc[0], gr[0], b0.x, b1.x, I.periodic[0], I.L[0], I.invL[0]) &&
                   ovl(gc[1], gr[1], b0.y, b1.y, I.periodic[1], I.L[1], I.invL[1]) &&
                   ovl(gc[2], gr[2], b0.z, b1.z, I.periodic[2], I.L[2], I.invL[2]);
        if (mode == WALK_FORCE) {
            // only subtrees holding buckets >= the group's first
            const int shift = I.logP - lvl;
            const int last = (int)(((nd + 1u) << shift) - 1u) - I.P;
            if (last < fl) return false;
            if (!gth) {
                gth = ovl(sc[0], sr[0], o0.x, o1.x, I.periodic[0], I.L[0], I.invL[0]) &&
                      ovl(sc[1], sr[1], o0.y, o1.y, I.periodic[1], I.L[1], I.invL[1]) &&
                      ovl(sc[2], sr[2], o0.z, o1.z, I.periodic[2], I.L[2], I.invL[2]);
            }
            if (lvl == I.logP && (int)(nd - I.P) < fl) gth = false;
        }
        return gth;
    };
    auto accept = [&](unsigned nd, int lvl) -> bool {
        const float4 b0 = tn[4 * nd], b1 = tn[4 * nd + 1];
        float4 o0 = b0, o1 = b1;
        if (mode == WALK_FORCE) {
            o0 = tn[4 * nd + 2];
            o1 = tn[4 * nd + 3];
        }
        return accept_b(nd, lvl, b0, b1, o0, o1);
    };
    // a group whose frontier or list outgrows kWalkCap (a particle with a
    // huge h, e.g. one leaving a free surface): the same warp tests every
    // leaf of the instance and writes the list to the shared overflow arena
    // behind the fixed per-group slots (two sweeps: count, write)
    auto exhaustive = [&]() {
        const unsigned lt = (1u << lane) - 1u;
        unsigned total = 0u;
        for (int base = 0; base < I.nb; base += 32) {
            const int k = base + lane;
            const bool acc = k < I.nb && accept((unsigned)(I.P + k), I.logP);
            total += __popc(__ballot_sync(kFull, acc));
        }
        unsigned off = 0u;
        if (lane == 0) off = atomicAdd(arena_used, total);
        off = __shfl_sync(kFull, off, 0);
        if ((unsigned long long)off + total > arena_cap) {
            if (lane == 0) {
                raise_status(st, ST_CAPACITY, g);
                list_cnt[g] = 0u;
                list_off[g] = (unsigned)g * kWalkCap;
            }
            return;
        }
        unsigned *out = list + (size_t)kp.ng * kWalkCap + off;
        unsigned pos = 0u;
        for (int base = 0; base < I.nb; base += 32) {
            const int k = base + lane;
            const bool acc = k < I.nb && accept((unsigned)(I.P + k), I.logP);
            const unsigned bal = __ballot_sync(kFull, acc);
            if (acc) out[pos + __popc(bal & lt)] = (unsigned)(I.boff + k);
            pos += __popc(bal);
        }
        if (lane == 0) {
            list_cnt[g] = total;
            list_off[g] = (unsigned)kp.ng * kWalkCap + off;
        }
    };
    // the frontier holds ACCEPTED nodes only: each round tests both children
    // of every accepted node and keeps the accepted ones (leaves become the
    // list as global bucket ids)
    unsigned *cur = buf[0], *nxt = buf[1];
    const int L0 = I.logP < 5 ? I.logP : 5;
    bool overflow = false;
    int ncur = 0;
    auto push = [&](bool acc, unsigned v, unsigned *dst, int &cnt) {
        const unsigned bal = __ballot_sync(kFull, acc);
        const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
        const int tot = cnt + __popc(bal);
        if (tot > kWalkCap) overflow = true;
        else if (acc) dst[pos] = v;
        cnt = min(tot, kWalkCap);
    };
    const bool top_leaf = L0 == I.logP;
    for (int base = 0; base < (1 << L0); base += 32) {
        const int k = base + lane;
        const unsigned nd = (1u << L0) + (unsigned)k;
        const bool acc = k < (1 << L0) && accept(nd, L0);
        push(acc, top_leaf ? (unsigned)I.boff + (nd - (unsigned)I.P) : nd, cur, ncur);
    }
    __syncwarp();
    // each round descends two levels where it can: the bounds of a node hold
    // those of its descendants, so testing the grandchildren of the accepted
    // nodes directly accepts the same nodes as two rounds of children tests,
    // with half the rounds of dependent loads.  Per round a lane loads four
    // nodes: two children of each of two frontier entries, or the four
    // grandchildren of one.
    for (int lvl = L0 + 1; lvl <= I.logP && !overflow;) {
        const int step = lvl < I.logP ? 2 : 1;
        const int tl = lvl + step - 1;  // level of the nodes tested
        const bool leaf = tl == I.logP;
        const int per = step == 2 ? 32 : 64;  // frontier entries per iteration
        int nnext = 0;
        for (int base = 0; base < ncur; base += per) {
            unsigned nd[4];
            bool have[4];
            float4 nb[4][4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int q = step == 2 ? 0 : (t >> 1);
                const int k = base + 32 * q + lane;
                have[t] = k < ncur;
                const unsigned par = have[t] ? cur[k] : 1u;
                nd[t] = step == 2 ? 4u * par + (unsigned)t : 2u * par + (unsigned)(t & 1);
                const float4 *cn = tn + 4 * (size_t)nd[t];
                nb[t][0] = cn[0];
                nb[t][1] = cn[1];
                if (mode == WALK_FORCE) {
                    nb[t][2] = cn[2];
                    nb[t][3] = cn[3];
                } else {
                    nb[t][2] = nb[t][0];
                    nb[t][3] = nb[t][1];
                }
            }
            bool acc[4];
#pragma unroll
            for (int t = 0; t < 4; ++t)
                acc[t] = have[t] && accept_b(nd[t], tl, nb[t][0], nb[t][1], nb[t][2], nb[t][3]);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (step == 1 && base + 32 * (t >> 1) >= ncur) break;  // (warp-uniform)
                push(acc[t], leaf ? (unsigned)I.boff + (nd[t] - (unsigned)I.P) : nd[t], nxt,
                     nnext);
            }
        }
        __syncwarp();
        unsigned *t = cur;
        cur = nxt;
        nxt = t;
        ncur = nnext;
        lvl += step;
    }
    if (overflow) {
        exhaustive();
        return;
    }
    unsigned *out = list + (size_t)g * kWalkCap;
    for (int k = lane; k < ncur; k += 32) out[k] = cur[k];
    if (lane == 0) {
        list_cnt[g] = (unsigned)ncur;
        list_off[g] = (unsigned)g * kWalkCap;
    }
}

__global__ void __launch_bounds__(128) k_walk(KParams kp, const Inst *__restrict__ insts,
                                              const int *__restrict__ gfirst,
                                              const int *__restrict__ bstart,
                                              const int *__restrict__ binst, int mode,
                                              const float4 *__restrict__ node,
                                              const float4 *__restrict__ pm,
                                              const int *__restrict__ origin,
                                              const float *__restrict__ h_walk,
                                              const unsigned *__restrict__ group_ids,
                                              const unsigned *__restrict__ group_cnt,
                                              unsigned *list, unsigned *list_cnt,
                                              unsigned *list_off, unsigned *arena_used,
                                              unsigned arena_cap, DevStatus *st)
{
    __shared__ unsigned buf[kWarpsPerBlock][2][kWalkCap];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gi0 = blockIdx.x * kWarpsPerBlock + wib;
    if (!group_ids) {  // every group, one warp each
        if (gi0 < kp.ng)
            walk_group(kp, insts, gfirst, bstart, binst, mode, node, pm, origin, h_walk, list,
                       list_cnt, list_off, arena_used, arena_cap, st, buf[wib], gi0, lane);
        return;
    }
    // the groups queued for a re-walk round, grid-stride over a small grid
    const int nq = (int)*group_cnt;
    for (int gi = gi0; gi < nq; gi += gridDim.x * kWarpsPerBlock)
        walk_group(kp, insts, gfirst, bstart, binst, mode, node, pm, origin, h_walk, list,
                   list_cnt, list_off, arena_used, arena_cap, st, buf[wib], (int)group_ids[gi],
                   lane);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_build(Ctx &c, const sph_particles &p, cudaStream_t s)
{
    const KParams &kp = c.kp;
    const int n = (int)p.n;
    int pr = prof_begin(c, s, SPH_PHASE_KEYS);
    // bounding boxes for the key quantisation (only open axes need data)
    if (kp.any_open) {
        k_bbox_partial<<<dim3(kBboxChunks, kp.ninst), 256, 0, s>>>(c.inst, p.x[0], p.x[1], p.x[2],
                                                                 c.bbox_part);
        c.launches += 1;
    }
    k_bbox_final<<<(kp.ninst + 127) / 128, 128, 0, s>>>(kp, c.inst, c.bbox_part, c.morton_box,
                                                        c.st);
    const int g = (n + 255) / 256;
    k_morton<<<g, 256, 0, s>>>(n, c.inst, c.pinst, p.x[0], p.x[1], p.x[2], c.morton_box,
                               c.keys[0], c.vals[0]);
    prof_end(c, s, pr);
    const int ntiles = (n + kSortTile - 1) / kSortTile;
    int cur = 0;
    pr = prof_begin(c, s, SPH_PHASE_SORT);
    for (int pass = 0; pass < kp.key_passes; ++pass) {
        const int shift = 8 * pass;
        k_sort_hist<<<ntiles, 256, 0, s>>>(c.keys[cur], n, shift, c.hist, ntiles);
        k_sort_rowscan<<<256, 1024, 0, s>>>(c.hist, ntiles, c.digit_tot);
        k_sort_scatter<<<ntiles, 256, 0, s>>>(c.keys[cur], c.vals[cur], c.keys[cur ^ 1],
                                              c.vals[cur ^ 1], n, shift, c.hist, c.digit_tot,
                                              ntiles);
        cur ^= 1;
    }
    prof_end(c, s, pr);
    const unsigned *perm = c.vals[cur];
    // permute every caller array through the scratch buffer
    typedef unsigned long long u64;
    PermFields pf;
    pf.f8[0] = (u64 *)p.x[0]; pf.f8[1] = (u64 *)p.x[1]; pf.f8[2] = (u64 *)p.x[2];
    pf.f8[3] = (u64 *)p.v[0]; pf.f8[4] = (u64 *)p.v[1]; pf.f8[5] = (u64 *)p.v[2];
    pf.f8[6] = (u64 *)p.u; pf.f8[7] = (u64 *)p.id;
    pf.f4[0] = p.m; pf.f4[1] = p.h; pf.f4[2] = p.rho; pf.f4[3] = p.omega;
    pf.f4[4] = p.a[0]; pf.f4[5] = p.a[1]; pf.f4[6] = p.a[2];
    pf.f4[7] = p.dudt_h; pf.f4[8] = p.dudt_av; pf.f4[9] = p.divv; pf.f4[10] = p.dt_i;
    pf.f2 = p.nngb;
    pf.f1 = p.iters;
    pf.f1b = p.mat;  // 112 B of scratch per particle hold every array
    pr = prof_begin(c, s, SPH_PHASE_PERMUTE);
    k_gather_all<<<g, 256, 0, s>>>(perm, n, pf, (char *)c.tmp);
    k_copyback_all<<<g, 256, 0, s>>>(n, pf, (const char *)c.tmp);
    prof_end(c, s, pr);
    if (c.mlp.record) {
        cudaError_t e = launch_mlp_permute(c, perm, n, s);
        if (e != cudaSuccess) return e;
    }
    if (c.rung) {  // hierarchical time steps: the rungs move with the particles
        cudaError_t e = launch_rung_permute(c, perm, n, s);
        if (e != cudaSuccess) return e;
    }
    // bucket layout on the sorted keys
    {
        const int tiles = (n + kPadTile - 1) / kPadTile;
        const unsigned long long *sk = c.keys[cur];
        const int gb = (kp.nb + 255) / 256;
        pr = prof_begin(c, s, SPH_PHASE_LAYOUT);
        k_pad_reduce<<<tiles, 256, 0, s>>>(n, c.inst, c.pinst, sk, p.h, c.morton_box, c.pad_agg);
        k_pad_scan<<<1, 1024, 0, s>>>(tiles, c.pad_agg);
        k_pad_init<<<gb, 256, 0, s>>>(kp.nb, c.inst, c.binst, c.bstart);
        k_pad_apply<<<tiles, 256, 0, s>>>(n, c.inst, c.pinst, sk, p.h, c.morton_box, c.pad_agg,
                                          c.bstart, c.pad_used);
        k_pad_fallback<<<gb, 256, 0, s>>>(kp.nb, c.inst, c.binst, c.pad_used, c.bstart);
        prof_end(c, s, pr);
        c.launches += 5;
    }
    // buckets and trees
    const int wb = (kp.nb * 32 + 127) / 128;
    pr = prof_begin(c, s, SPH_PHASE_BUCKETS);
    k_buckets<<<wb, 128, 0, s>>>(kp, c.inst, c.bstart, c.binst, p.x[0], p.x[1], p.x[2], p.m, p.h,
                                 c.origin, c.pm, c.ipos, c.pmd, c.node, 1, c.st);
    prof_end(c, s, pr);
    c.launches += 2 + 3 * kp.key_passes + 2 + 1;
    pr = prof_begin(c, s, SPH_PHASE_TREE);
    tree_refit(c, s, 0);
    prof_end(c, s, pr);
    return cudaGetLastError();
}

cudaError_t launch_refit(Ctx &c, const sph_particles &p, cudaStream_t s)
{
    const KParams &kp = c.kp;
    const int wb = (kp.nb * 32 + 127) / 128;
    c.launches += 1;
    int pr = prof_begin(c, s, SPH_PHASE_BUCKETS);
    k_buckets<<<wb, 128, 0, s>>>(kp, c.inst, c.bstart, c.binst, p.x[0], p.x[1], p.x[2], p.m, p.h,
                                 c.origin, c.pm, c.ipos, c.pmd, c.node, 2, c.st);
    prof_end(c, s, pr);
    pr = prof_begin(c, s, SPH_PHASE_TREE);
    tree_refit(c, s, 0);
    prof_end(c, s, pr);
    return cudaGetLastError();
}

// the leaves' boxes of balls were written by the density kernel (each warp
// for its bucket, with the new h); the upper levels follow here
cudaError_t launch_bob_refit(Ctx &c, const sph_particles &p, cudaStream_t s)
{
    (void)p;
    const int pr = prof_begin(c, s, SPH_PHASE_BOB_REFIT);
    tree_refit(c, s, 1);
    prof_end(c, s, pr);
    return cudaGetLastError();
}

cudaError_t launch_walk(Ctx &c, const sph_particles &p, int mode, int round, const float *h_walk,
                        cudaStream_t s)
{
    (void)p;
    const KParams &kp = c.kp;
    if (kp.ng <= 0) return cudaSuccess;
    const unsigned *ids = round < 0 ? nullptr : c.redo + (size_t)round * kp.ng;
    const unsigned *cnt = round < 0 ? nullptr : &c.st->redo_cnt[round];
    int g = (kp.ng + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (round >= 0 && g > kRoundBlocks) g = kRoundBlocks;
    // the overflow arena is emptied when every list is rebuilt
    if (round < 0) cudaMemsetAsync(c.arena_used, 0, sizeof(unsigned), s);
    c.launches += 1;
    const int pr = prof_begin(c, s, SPH_PHASE_WALK);
    k_walk<<<g, 32 * kWarpsPerBlock, 0, s>>>(kp, c.inst, c.gfirst, c.bstart, c.binst, mode, c.node,
                                             c.pm, c.origin, h_walk, ids, cnt, c.list, c.list_cnt,
                                             c.list_off, c.arena_used, (unsigned)c.arena_cap,
                                             c.st);
    prof_end(c, s, pr);
    return cudaGetLastError();
}

cudaError_t launch_walk_queue(Ctx &c, int mode, const unsigned *ids, const unsigned *cnt,
                              const float *h_walk, cudaStream_t s)
{
    const KParams &kp = c.kp;
    if (kp.ng <= 0) return cudaSuccess;
    // a queue that may hold every group: one warp slot per group, the
    // surplus warps leave at once
    const int g = (kp.ng + kWarpsPerBlock - 1) / kWarpsPerBlock;
    cudaMemsetAsync(c.arena_used, 0, sizeof(unsigned), s);
    c.launches += 1;
    const int pr = prof_begin(c, s, SPH_PHASE_WALK);
    k_walk<<<g, 32 * kWarpsPerBlock, 0, s>>>(kp, c.inst, c.gfirst, c.bstart, c.binst, mode, c.node,
                                             c.pm, c.origin, h_walk, ids, cnt, c.list, c.list_cnt,
                                             c.list_off, c.arena_used, (unsigned)c.arena_cap,
                                             c.st);
    prof_end(c, s, pr);
    return cudaGetLastError();
}

}  // namespace sph
