// DAFMM application on the device (Section 5, steps 3-6).
//
// Every tree pass is a block-sparse complex matrix-vector product between
// coefficient spaces (P2M, M2M and directional M2M up; M2L and directional
// M2L across; directional L2L, L2L down).  The blocks of one output row are
// stored contiguously at their realised NCA ranks, so a row is one
// rout x J column-major matrix, read exactly once per application: the
// single-right-hand-side apply is bound by HBM bandwidth (complex64) or by
// the FP64 pipes (complex128).
//
// Streaming: rows are cut into column ranges ("chunks") of about 1536
// entries.  Each warp runs a two-stage pipeline: one lane issues a TMA bulk
// copy (cp.async.bulk, completion on an mbarrier) of the next chunk's matrix
// into shared memory while the warp gathers the chunk's input coefficients
// and multiplies the current stage (lanes cover the output index and, for
// narrow blocks, interleave the columns).  Every mbarrier wait is bounded; on
// timeout the kernel raises a device error flag, drains its own copy in
// flight and returns.  A chunk that is its row's only chunk writes the row;
// otherwise it writes a partial that a second kernel adds in a fixed order,
// so results are bit-reproducible.  The M2L of all levels is one launch.
// The leaf kernel fuses L2P, the tabulated near field (nine shared 16 x 16
// blocks in shared memory) and the epilogue v + kappa^2 q (.).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <unordered_map>
#include <mutex>
#include <string>

#include "ops.h"

namespace dafmm {
namespace {

template <typename T>
struct V2;
template <>
struct V2<double> {
    using t = double2;
};
template <>
struct V2<float> {
    using t = float2;
};

constexpr int kMaxPass = 24;        // passes in one launch group
constexpr int kMaxPhase = 32;       // phases of the fused single-right-hand-side launch
constexpr int kMaxRhs = 64;         // right-hand sides of one application
constexpr int kFlagDirectHost = 1 << 8;  // same bits as the device-side record flags
constexpr int kFlagAddHost = 1 << 9;
constexpr long kChunkElems = 1024;    // matrix entries per chunk (8 KB in complex64)
constexpr long kChunkElems64 = 512;   // per chunk of the single-right-hand-side complex128 launch (8 KB)

template <typename T>
struct PassArgs {
    const int* rout;    // per row
    const long* rbase;  // per row: element offset of the row's matrix in mats
    const int* cbase;   // per row: offset of the row's columns in xmap
    const int* xmap;    // per column: index of its input coefficient in x
    const typename V2<T>::t* mats;
    const typename V2<T>::t* x;
    const typename V2<T>::t* x2;  // fused launch: second input added to x (locals from the parent), or null
    const double2* xd;            // fused launch: complex128 input read instead of x (the vector itself), or null
    typename V2<T>::t* y;
    int ldy;
};

// Schedule of the fused launch: phases of the chunk list and the pass
// dependencies (see Fused in ops.h).
struct Sched {
    // chain list: the passes without slack, phase by phase, in static warp shares
    int nph;
    int base[kMaxPhase + 1];    // first chunk of each phase; base[nph] = chain chunks
    int kpw[kMaxPhase];         // chunks per warp in each phase
    int sbase[kMaxPhase];       // warp shares in the phases before (partial slots)
    unsigned phdeps[kMaxPhase]; // passes read by the passes of each phase
    int wlo[kMaxPhase];         // the warps sharing each phase: wlo .. wlo + wn - 1, in the
    int wn[kMaxPhase];          // order (warp of its CTA, CTA)
    int chain_split;            // the chain has warps of its own: they take no pieces
    // bulk list: the passes with slack, cut into pieces handed out in order
    int npieces;
    const int4* pieces;         // per piece: {first chunk, end chunk, partial slot, pass}
    int* next_piece;            // piece counter
    unsigned deps[kMaxPass];    // per pass: passes whose rows it reads
    int target[kMaxPass];       // per pass: rows it writes
    int dphase[kMaxPass];       // per pass: latest phase among the passes it reads (-1: none)
    unsigned pub;               // passes read by another pass of the launch: the only ones counted
    // static tables the launch reads (chunk records, column maps), prefetched
    // into L2 at the start: the operators stream past them evict_first
    const char* pf_ptr[kMaxPass + 1];
    int pf_bytes[kMaxPass + 1];
    int npf;
};

template <typename T>
struct GroupArgs {
    PassArgs<T> p[kMaxPass];
};

template <typename T>
__device__ __forceinline__ void cmac(T& ar, T& ai, typename V2<T>::t m, typename V2<T>::t x)
{
    ar = fma(m.x, x.x, fma(-m.y, x.y, ar));
    ai = fma(m.x, x.y, fma(m.y, x.x, ai));
}

constexpr int kMaxChunkCols = 128;   // columns per chunk (shared gather buffer)
constexpr int kStreamWarps = 4;      // warps per CTA, each with its own pipeline
constexpr long kSpinLimit = 1L << 22;  // bounded mbarrier waits

template <typename T>
struct StreamCfg {
    using C = typename V2<T>::t;
    // complex128 chunks hold half as many entries, so that three CTAs fit an SM
    static constexpr long kElems = sizeof(T) == 8 ? kChunkElems64 : kChunkElems;
    static constexpr int kStage = ((int)(kElems * sizeof(C)) + 32 + 127) / 128 * 128;
    static constexpr int kXs = kMaxChunkCols * (int)sizeof(C);
    static constexpr int kWarp = 2 * kStage + kXs + 128;  // two stages, gather buffer, barriers
    static constexpr int kCta = kStreamWarps * kWarp;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Arm the barrier for bytes and start one bulk copy global -> shared.
__device__ __forceinline__ void tma_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// The same with an L2 cache policy (evict_first for data read once).
__device__ __forceinline__ void tma_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar, unsigned long long pol)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
                 : "memory");
}

// Wait for the barrier's phase with the given parity; false after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity)
{
    const unsigned a = smem_u32(bar);
    for (long k = 0; k < kSpinLimit; k++) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// A chunk record is two int4: a = {pass | direct << 8 | rout << 16, row,
// ncol, first xmap index}, b = {element offset of the chunk's matrix (lo, hi),
// entries, first chunk of the row}.  The matrix of a chunk is ld x ncol
// (ld = rout rounded up to even) and starts at an even element, so its bytes
// start 16-byte aligned.
constexpr int kMaxPrefetch = kMaxChunkCols / 32;

template <typename T>
__device__ __forceinline__ const char* chunk_src(const GroupArgs<T>& g, const int4& a, const int4& b, unsigned& bytes)
{
    using C = typename V2<T>::t;
    const PassArgs<T>& pa = g.p[a.x & 0xff];
    const long elem = (long)(unsigned)b.x | ((long)b.y << 32);
    const int ro = (a.x >> 16) & 0xffff;
    bytes = (unsigned)((size_t)a.z * (ro + (ro & 1)) * sizeof(C));
    return (const char*)(pa.mats + elem);
}

// Record flags (bits of a.x above the pass index).
constexpr int kFlagDirect = 1 << 8;  // the row's only chunk: write y itself
constexpr int kFlagAdd = 1 << 9;     // add to y (it already holds this application's values)

// Partial slots of a row split over chunks [c0, c1) of a list whose chunk
// ranges start at base + m * kpw: c0 and every range start inside (c0, c1),
// one per range that touches the row.
__host__ __device__ __forceinline__ int row_slots(int c0, int c1, int base, int kpw)
{
    return 1 + ((c1 - 1 - base) / kpw - (c0 - base) / kpw);
}
__device__ __forceinline__ int next_slot(int c, int base, int kpw) { return base + ((c - base) / kpw + 1) * kpw; }

__device__ __forceinline__ int atom_add_acq_rel(int* p, int v)
{
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void red_add_release(int* p, int v)
{
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

constexpr int kDoneStride = 32;  // ints between two pass counters: one 128-byte line each

// Publish n finished rows of a pass: the rows' stores (ordered before lane 0
// by the barrier) become visible at device scope before the pass's row
// counter moves (release).
__device__ __forceinline__ void rows_done(int* done, int pass, int n, int lane)
{
    __syncwarp();
    if (lane == 0) red_add_release(&done[pass * kDoneStride], n);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long kDepWaitNs = 200000000ull;  // a wait on another pass gives up after 0.2 s
constexpr long kDepSpinLimit = 1L << 24;                   // and after this many polls in any case

// Wait until every pass in `need` has written all its rows (`ready` caches
// the passes already seen complete): 1, or -1 when a wait gave up.  Lane 0
// polls with acquire semantics and a growing back-off; the barrier after it
// orders the other lanes' later loads.
__device__ __forceinline__ int deps_wait(const Sched& sc, const int* done, unsigned need, unsigned& ready, int lane)
{
    unsigned todo = need & ~ready;
    while (todo) {
        const int q = __ffs(todo) - 1;
        int ok = 1;
        if (lane == 0) {
            const unsigned long long t0 = global_ns();
            unsigned nap = 32;
            for (long k = 0; ld_acquire(&done[q * kDoneStride]) < sc.target[q]; k++) {
                if (k >= kDepSpinLimit || global_ns() - t0 > kDepWaitNs) {
                    ok = -1;
                    break;
                }
                __nanosleep(nap);
                nap = nap < 512 ? 2 * nap : nap;
            }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (ok < 0) return -1;
        ready |= 1u << q;
        todo &= todo - 1;
    }
    __syncwarp();
    return 1;
}

// Complex128 coefficients of the single-right-hand-side launch are kept as
// float pairs {re hi, im hi, re lo, im lo} in the 16 bytes of a double2
// (double-float arithmetic; see Acc<double>).
__device__ __forceinline__ float4 as_df(double2 d)
{
    union {
        double2 d;
        float4 f;
    } u;
    u.d = d;
    return u.f;
}
__device__ __forceinline__ double2 df_bits(float4 f)
{
    union {
        double2 d;
        float4 f;
    } u;
    u.f = f;
    return u.d;
}

// (h, l) = a + b for float pairs (two-sum of the high words, the low words
// and the error added, renormalised).
__device__ __forceinline__ void df_add(float& h, float& l, float ah, float al, float bh, float bl)
{
    const float s = __fadd_rn(ah, bh);
    const float v = __fsub_rn(s, ah);
    const float e = __fadd_rn(__fadd_rn(__fsub_rn(ah, __fsub_rn(s, v)), __fsub_rn(bh, v)), __fadd_rn(al, bl));
    h = __fadd_rn(s, e);
    l = __fsub_rn(e, __fsub_rn(h, s));
}

__device__ __forceinline__ float4 df4_add(float4 a, float4 b)
{
    float4 r;
    df_add(r.x, r.z, a.x, a.z, b.x, b.z);
    df_add(r.y, r.w, a.y, a.w, b.y, b.w);
    return r;
}

// A double as a float pair: hi its nearest float, lo the nearest float of the rest.
__device__ __forceinline__ double2 df_split(double2 v)
{
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    return df_bits(make_float4(rh, ih, __double2float_rn(v.x - (double)rh), __double2float_rn(v.y - (double)ih)));
}

// o + p[0] + p[Pld] + ... + p[(n - 1) Pld], added in that order; the
// partials are loaded a batch at a time, so that their latencies overlap
// (the 16-byte float pairs one at a time: batches of them measured slower).
template <typename T>
__device__ __forceinline__ typename V2<T>::t sum_partials(typename V2<T>::t o, const typename V2<T>::t* p, int Pld, int n)
{
    using C = typename V2<T>::t;
    constexpr int kSumBatch = sizeof(T) == 8 ? 1 : 8;
    for (int q = 0; q < n; q += kSumBatch) {
        C v[kSumBatch];
#pragma unroll
        for (int u = 0; u < kSumBatch; u++)
            if (q + u < n) v[u] = __ldcg(&p[(size_t)(q + u) * Pld]);
#pragma unroll
        for (int u = 0; u < kSumBatch; u++)
            if (q + u < n) {
                if constexpr (sizeof(T) == 8) {
                    o = df_bits(df4_add(as_df(o), as_df(v[u])));  // float pairs (double-float)
                } else {
                    o.x += v[u].x;
                    o.y += v[u].y;
                }
            }
    }
    return o;
}

// Partial slot of the warp share of phase k that starts at chunk c.
__device__ __forceinline__ int share_slot(const Sched& sc, int k, int c) { return sc.sbase[k] + (c - sc.base[k]) / sc.kpw[k]; }

// A split row [c0, c1) of phase k.  Each warp whose share starts inside the
// row (and so began with it) writes its partial to its share's slot and
// counts in, without waiting (put_partial).  The owner, the warp whose share
// holds c0 (the row is the last of its share), has written its own part to
// y; it waits for the others' partials (bounded), adds them to y in share
// order, so that the result does not depend on timing, and re-arms the
// counter (own_row; false when the wait gave up).
__device__ __forceinline__ void put_partial(int* cnt, int c0, int lane)
{
    // the partial's stores come before lane 0's release: the barrier orders
    // them, the release is cumulative
    __syncwarp();
    if (lane == 0) red_add_release(&cnt[c0], 1);
}

template <typename T>
__device__ __forceinline__ bool own_row(typename V2<T>::t* y, const typename V2<T>::t* P, int Pld, int* cnt, int c0, int c1,
                                        const Sched& sc, int k, int ro, int lane)
{
    using C = typename V2<T>::t;
    const int base = sc.base[k], kpw = sc.kpw[k];
    const int others = row_slots(c0, c1, base, kpw) - 1;
    int ok = 1;
    if (lane == 0) {
        const unsigned long long t0 = global_ns();
        unsigned nap = 32;
        for (long n = 0; ld_acquire(&cnt[c0]) < others; n++) {
            if (n >= kDepSpinLimit || global_ns() - t0 > kDepWaitNs) {
                ok = 0;
                break;
            }
            __nanosleep(nap);
            nap = nap < 512 ? 2 * nap : nap;
        }
        if (ok) cnt[c0] = 0;
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return false;
    __syncwarp();  // lane 0's acquire, and the owner's own stores to y, come before every lane's reads
    // the shares that start inside the row hold consecutive slots, in share order
    const int s1 = share_slot(sc, k, next_slot(c0, base, kpw));
    for (int i = lane; i < ro; i += 32) y[i] = sum_partials<T>(y[i], P + (size_t)s1 * Pld + i, Pld, others);
    return true;
}

// Indices (into x) of the input coefficients of the chunk described by a.
template <typename T>
__device__ __forceinline__ void gather_idx(const GroupArgs<T>& g, const int4& a, int lane, int* xi)
{
    const PassArgs<T>& pa = g.p[a.x & 0xff];
#pragma unroll
    for (int k = 0; k < kMaxPrefetch; k++) {
        const int t = lane + 32 * k;
        if (t < a.z) xi[k] = pa.xmap[a.w + t];
    }
}

// Load (into registers) the input coefficients at indices xi.  Coefficients
// written earlier in the same launch are read through L2.
template <typename T>
__device__ __forceinline__ void gather_val(const GroupArgs<T>& g, const int4& a, int lane, const int* xi, typename V2<T>::t* xr)
{
    using C = typename V2<T>::t;
    const PassArgs<T>& pa = g.p[a.x & 0xff];
#pragma unroll
    for (int k = 0; k < kMaxPrefetch; k++) {
        const int t = lane + 32 * k;
        if (t < a.z) {
            const int ix = xi[k];
            C v;
            if constexpr (sizeof(T) == 8) {
                // complex128: float pairs (the input split, coefficients stored so)
                if (pa.xd) {
                    v = df_split(pa.xd[ix]);
                } else {
                    v = __ldcg(pa.x + ix);
                    if (pa.x2) v = df_bits(df4_add(as_df(v), as_df(__ldcg(pa.x2 + ix))));
                }
            } else if (pa.xd) {
                const double2 d = pa.xd[ix];
                v.x = (T)d.x;
                v.y = (T)d.y;
            } else {
                v = __ldcg(pa.x + ix);
                if (pa.x2) {
                    const C u = __ldcg(pa.x2 + ix);
                    v.x += u.x;
                    v.y += u.y;
                }
            }
            xr[k] = v;
        }
    }
}

// Per-lane accumulators of one output row: 4 slots x (re, im), two
// independent sets (A for even, B for odd column steps).
template <typename T>
struct Acc {
    T r[2][4], i[2][4];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int s = 0; s < 2; s++)
#pragma unroll
            for (int k = 0; k < 4; k++) r[s][k] = i[s][k] = 0;
    }
};

// Complex128 in the single-right-hand-side launch is carried in float pairs
// (hi + lo, about 48 significant bits): FP64 instructions issue at 1/64 of
// the FP32 rate on GB300, so the products and sums of a chunk run in FP32
// with exact error terms (double-float arithmetic); the pass outputs stay
// float pairs too (the leaf kernel rounds them to double).  Matrices come as
// float4 {re hi, im hi, re lo, im lo} (the same 16 bytes as a double2); the
// input vector is split when it is gathered.
template <>
struct Acc<double> {
    float rh[2][4], rl[2][4], ih[2][4], il[2][4];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int s = 0; s < 2; s++)
#pragma unroll
            for (int k = 0; k < 4; k++) rh[s][k] = rl[s][k] = ih[s][k] = il[s][k] = 0.f;
    }
};

// (sh, sl) += a b for float pairs a = ah + al, b = bh + bl: the rounding
// error of ah bh exactly (FMA), the cross terms, and a two-sum into sh whose
// error goes to sl.  Explicitly rounded operations keep the compiler from
// contracting the error-free steps.
__device__ __forceinline__ void df_mac(float& sh, float& sl, float ah, float al, float bh, float bl)
{
    const float p = __fmul_rn(ah, bh);
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float t = __fadd_rn(sh, p);
    const float v = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, v)), __fsub_rn(p, v));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(err, e));
}

// (re, im) += m x for complex float pairs {re hi, im hi, re lo, im lo}.
__device__ __forceinline__ void df_cmac(float& rh, float& rl, float& ih, float& il, float4 m, float4 x)
{
    df_mac(rh, rl, m.x, m.z, x.x, x.z);
    df_mac(rh, rl, -m.y, -m.w, x.y, x.w);
    df_mac(ih, il, m.x, m.z, x.y, x.w);
    df_mac(ih, il, m.y, m.w, x.x, x.z);
}

// Multiply one chunk held in shared memory into the accumulators.
// complex64: lane handles row pairs (2p, 2p+1) with 16-byte loads, p = lane %
// NP (+32); complex128: lane handles rows i = lane % ro (+32k).  When the
// rows fit in fewer than 32 lanes, lane groups jp interleave the columns.
template <typename T>
__device__ __forceinline__ void chunk_mac(Acc<T>& acc, const typename V2<T>::t* M, const typename V2<T>::t* xs, int ro, int ld,
                                          int ncol, int lane)
{
    if constexpr (sizeof(T) == 4) {
        const int NP = (ro + 1) >> 1;
        if (NP <= 32) {
            const int JP = 32 / NP, p = lane % NP, jp = lane / NP;
            if (jp >= JP) return;
            const float4* M4 = (const float4*)(M) + p;
            const int ld2 = ld >> 1;
            int j = jp;
#pragma unroll 2
            for (; j + JP < ncol; j += 2 * JP) {
                const float4 m0 = M4[j * ld2], m1 = M4[(j + JP) * ld2];
                const float2 x0 = xs[j], x1 = xs[j + JP];
                acc.r[0][0] = fmaf(m0.x, x0.x, fmaf(-m0.y, x0.y, acc.r[0][0]));
                acc.i[0][0] = fmaf(m0.x, x0.y, fmaf(m0.y, x0.x, acc.i[0][0]));
                acc.r[0][1] = fmaf(m0.z, x0.x, fmaf(-m0.w, x0.y, acc.r[0][1]));
                acc.i[0][1] = fmaf(m0.z, x0.y, fmaf(m0.w, x0.x, acc.i[0][1]));
                acc.r[1][0] = fmaf(m1.x, x1.x, fmaf(-m1.y, x1.y, acc.r[1][0]));
                acc.i[1][0] = fmaf(m1.x, x1.y, fmaf(m1.y, x1.x, acc.i[1][0]));
                acc.r[1][1] = fmaf(m1.z, x1.x, fmaf(-m1.w, x1.y, acc.r[1][1]));
                acc.i[1][1] = fmaf(m1.z, x1.y, fmaf(m1.w, x1.x, acc.i[1][1]));
            }
            if (j < ncol) {
                const float4 m0 = M4[j * ld2];
                const float2 x0 = xs[j];
                acc.r[0][0] = fmaf(m0.x, x0.x, fmaf(-m0.y, x0.y, acc.r[0][0]));
                acc.i[0][0] = fmaf(m0.x, x0.y, fmaf(m0.y, x0.x, acc.i[0][0]));
                acc.r[0][1] = fmaf(m0.z, x0.x, fmaf(-m0.w, x0.y, acc.r[0][1]));
                acc.i[0][1] = fmaf(m0.z, x0.y, fmaf(m0.w, x0.x, acc.i[0][1]));
            }
        } else {
            const float4* M4 = (const float4*)(M);
            const int ld2 = ld >> 1;
            const bool second = lane + 32 < NP;
#pragma unroll 2
            for (int j = 0; j < ncol; j++) {
                const float2 x0 = xs[j];
                const float4 m0 = M4[j * ld2 + lane];
                acc.r[0][0] = fmaf(m0.x, x0.x, fmaf(-m0.y, x0.y, acc.r[0][0]));
                acc.i[0][0] = fmaf(m0.x, x0.y, fmaf(m0.y, x0.x, acc.i[0][0]));
                acc.r[0][1] = fmaf(m0.z, x0.x, fmaf(-m0.w, x0.y, acc.r[0][1]));
                acc.i[0][1] = fmaf(m0.z, x0.y, fmaf(m0.w, x0.x, acc.i[0][1]));
                if (second) {
                    const float4 m1 = M4[j * ld2 + lane + 32];
                    acc.r[0][2] = fmaf(m1.x, x0.x, fmaf(-m1.y, x0.y, acc.r[0][2]));
                    acc.i[0][2] = fmaf(m1.x, x0.y, fmaf(m1.y, x0.x, acc.i[0][2]));
                    acc.r[0][3] = fmaf(m1.z, x0.x, fmaf(-m1.w, x0.y, acc.r[0][3]));
                    acc.i[0][3] = fmaf(m1.z, x0.y, fmaf(m1.w, x0.x, acc.i[0][3]));
                }
            }
        }
    } else {
        // float pairs (see Acc<double>): M and xs hold float4 entries
        const float4* M4 = (const float4*)M;
        const float4* X4 = (const float4*)xs;
        if (ro <= 32) {
            // two column streams per lane (sets 0/1)
            const int JP = 32 / ro, i = lane % ro, jp = lane / ro;
            if (jp >= JP) return;
            const float4* Mi = M4 + i;
            int j = jp;
            for (; j + JP < ncol; j += 2 * JP) {
                const float4 m0 = Mi[j * ld], m1 = Mi[(j + JP) * ld];
                const float4 x0 = X4[j], x1 = X4[j + JP];
                df_cmac(acc.rh[0][0], acc.rl[0][0], acc.ih[0][0], acc.il[0][0], m0, x0);
                df_cmac(acc.rh[1][0], acc.rl[1][0], acc.ih[1][0], acc.il[1][0], m1, x1);
            }
            if (j < ncol) df_cmac(acc.rh[0][0], acc.rl[0][0], acc.ih[0][0], acc.il[0][0], Mi[j * ld], X4[j]);
        } else {
            // rows lane + 32 k; even columns into set 0, odd into set 1
            const int nck = (ro + 31) / 32;
            int j = 0;
            for (; j + 1 < ncol; j += 2) {
                const float4 x0 = X4[j], x1 = X4[j + 1];
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if (k < nck && k * 32 + lane < ro) {
                        const float4 m0 = M4[j * ld + k * 32 + lane], m1 = M4[(j + 1) * ld + k * 32 + lane];
                        df_cmac(acc.rh[0][k], acc.rl[0][k], acc.ih[0][k], acc.il[0][k], m0, x0);
                        df_cmac(acc.rh[1][k], acc.rl[1][k], acc.ih[1][k], acc.il[1][k], m1, x1);
                    }
            }
            if (j < ncol) {
                const float4 x0 = X4[j];
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if (k < nck && k * 32 + lane < ro)
                        df_cmac(acc.rh[0][k], acc.rl[0][k], acc.ih[0][k], acc.il[0][k], M4[j * ld + k * 32 + lane], x0);
            }
        }
    }
}

// Sum the accumulators over the lane groups and write the row (to y when the
// chunk range covers the whole row, else to the partial slot P[pslot]).
// Complex128 rows are written as float pairs (double-float, see Acc<double>).
__device__ __forceinline__ void flush_row_df(Acc<double>& acc, int ro, int lane, double2* dst, bool to_y, int accumulate)
{
    float h[4], l[4], ih[4], il[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        df_add(h[k], l[k], acc.rh[0][k], acc.rl[0][k], acc.rh[1][k], acc.rl[1][k]);
        df_add(ih[k], il[k], acc.ih[0][k], acc.il[0][k], acc.ih[1][k], acc.il[1][k]);
    }
    auto put = [&](int row, float rh, float rl, float jh, float jl) {
        float4 v = make_float4(rh, jh, rl, jl);
        if (to_y && accumulate) v = df4_add(v, as_df(dst[row]));
        dst[row] = df_bits(v);
    };
    if (ro <= 32) {
        const int JP = 32 / ro, i = lane % ro, jp = lane / ro;
        for (int q = 1; q < JP; q++) {
            const int src = (lane + q * ro) & 31;
            const float th = __shfl_sync(0xffffffffu, h[0], src), tl = __shfl_sync(0xffffffffu, l[0], src);
            const float uh = __shfl_sync(0xffffffffu, ih[0], src), ul = __shfl_sync(0xffffffffu, il[0], src);
            if (jp == 0) {
                df_add(h[0], l[0], h[0], l[0], th, tl);
                df_add(ih[0], il[0], ih[0], il[0], uh, ul);
            }
        }
        if (jp == 0) put(i, h[0], l[0], ih[0], il[0]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (k * 32 + lane < ro) put(k * 32 + lane, h[k], l[k], ih[k], il[k]);
    }
}

template <typename T>
__device__ __forceinline__ void flush_row(Acc<T>& acc, int ro, int lane, typename V2<T>::t* dst, bool to_y, int accumulate)
{
    using C = typename V2<T>::t;
    if constexpr (sizeof(T) == 8) {
        flush_row_df(acc, ro, lane, dst, to_y, accumulate);
    } else {
        // combine the two independent sets
        T r0[4], i0[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            r0[k] = acc.r[0][k] + acc.r[1][k];
            i0[k] = acc.i[0][k] + acc.i[1][k];
        }
        auto put = [&](int row, T re, T im) {
            C* q = dst + row;
            if (to_y && accumulate) {
                const C o = *q;
                re += o.x;
                im += o.y;
            }
            C r;
            r.x = re;
            r.y = im;
            *q = r;
        };
        const int NP = (ro + 1) >> 1;
        if (NP <= 32) {
            const int JP = 32 / NP, p = lane % NP, jp = lane / NP;
#pragma unroll
            for (int k = 0; k < 2; k++)
                for (int q = 1; q < JP; q++) {
                    const int src = (lane + q * NP) & 31;
                    const float tr = __shfl_sync(0xffffffffu, r0[k], src);
                    const float ti = __shfl_sync(0xffffffffu, i0[k], src);
                    if (jp == 0) {
                        r0[k] += tr;
                        i0[k] += ti;
                    }
                }
            if (jp == 0) {
                put(2 * p, r0[0], i0[0]);
                if (2 * p + 1 < ro) put(2 * p + 1, r0[1], i0[1]);
            }
        } else {
            put(2 * lane, r0[0], i0[0]);
            if (2 * lane + 1 < ro) put(2 * lane + 1, r0[1], i0[1]);
            if (lane + 32 < NP) {
                put(2 * lane + 64, r0[2], i0[2]);
                if (2 * lane + 65 < ro) put(2 * lane + 65, r0[3], i0[3]);
            }
        }
    }
}

// A warp's share of one chain phase: chunks [b, e), the next to schedule c.
struct Slice {
    int k, b, c, e;
};

// First non-empty share of warp w (in the order of Sched::wlo) in chain
// phases k, k+1, ...
__device__ __forceinline__ bool slice_from(const Sched& sc, int k, int w, Slice& sl)
{
    for (; k < sc.nph; k++) {
        const int sh = w - sc.wlo[k];
        if (sh < 0 || sh >= sc.wn[k]) continue;
        const int b = sc.base[k] + sh * sc.kpw[k];
        const int e = min(sc.base[k + 1], b + sc.kpw[k]);
        if (b < e) {
            sl.k = k;
            sl.b = b;
            sl.c = b;
            sl.e = e;
            return true;
        }
    }
    return false;
}

constexpr int kPiece = 4;  // chunks per bulk piece

// Warps given to the chain phases after the first: this many times the
// chain's share of the chunks after the first phase (the rest stream the
// slack passes); the chain's dependent steps need the margin.
constexpr double kChainShare64 = 1.4, kChainShare128 = 1.0;
// Plans: the slack passes as pieces taken in order (else in phases of their
// own), and the chain phases after the first on their own warps.
constexpr bool kPieces128 = true, kSplit128 = true;
constexpr bool kPieces64 = false, kSplit64 = true;
constexpr bool kDedupChunks = true;  // equal chunks of a pass share one copy of their matrix

// One scheduled chunk: c (-1: none); kind 0: chain (aux = phase, end = the
// share's end), 1: bulk (aux = the piece's partial slot, end = the piece's end).
struct Item {
    int c, kind, aux, end;
};

__device__ __forceinline__ int ld_relaxed(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int4 shfl4(int4 v)
{
    v.x = __shfl_sync(0xffffffffu, v.x, 0);
    v.y = __shfl_sync(0xffffffffu, v.y, 0);
    v.z = __shfl_sync(0xffffffffu, v.z, 0);
    v.w = __shfl_sync(0xffffffffu, v.w, 0);
    return v;
}

// A piece of a bulk row [c0, c1) (pieces start at c0 + m kPiece) has left its
// partial in slot `slot`; the last piece to finish sums the row's partials in
// piece order into y (so the result does not depend on timing) and re-arms
// the counter.  True in the warp that wrote y.
template <typename T>
__device__ __forceinline__ bool bulk_finish(typename V2<T>::t* y, const typename V2<T>::t* P, int Pld, int* cnt, int c0, int c1, int slot,
                                            int c, int ro, int lane)
{
    using C = typename V2<T>::t;
    const int np = (c1 - c0 + kPiece - 1) / kPiece;
    const int s0 = slot - (c - c0) / kPiece;
    __syncwarp();
    int last = 0;
    if (lane == 0) last = atom_add_acq_rel(&cnt[c0], 1) + 1 == np;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return false;
    __syncwarp();
    for (int i = lane; i < ro; i += 32) {
        const C* p = P + (size_t)s0 * Pld + i;
        if constexpr (sizeof(T) == 8) {
            y[i] = sum_partials<T>(__ldcg(p), p + Pld, Pld, np - 1);
        } else {
            C z;
            z.x = 0;
            z.y = 0;
            y[i] = sum_partials<T>(z, p, Pld, np);
        }
    }
    if (lane == 0) cnt[c0] = 0;
    return true;
}

// Every tree pass of one application.  The chunk list is cut into phases,
// each shared out in static, contiguous shares to a range of warps
// (Sched::wlo, wn): phase 0 to every warp; with the chain split, the later
// chain phases to the first warps and, in the static plan, each slack M2L
// pass as a phase of its own to the others.  In the dynamic plan the slack
// passes are instead pieces of kPiece chunks taken in order from a counter:
// at the end of a unit (a share or a piece) a warp takes the next chain
// share when the passes it reads are complete, else the next piece when its
// inputs are complete, else whichever reads the earlier phase; with the
// chain split, chain warps take no pieces.  The choice is made two chunks
// ahead, so every chunk's matrix is copied in (TMA, two stages) before it is
// needed.  Readiness is polled with relaxed loads issued an iteration early;
// the first chunk of a pass waits (bounded) on its inputs' row counters with
// acquire semantics.  Split rows of a phase are summed by the warp that
// holds their first chunk, split rows of pieces by their last piece, both in
// a fixed order.  A warp counts its finished rows of a pass in its pass's
// counter with one release when its run of chunks of that pass ends, and
// before it waits on anything; a pass is complete only when every run of it
// is, so the count arrives no later than it would row by row, and a waiting
// warp holds no uncounted rows.  Passes that no other pass of the launch
// reads are not counted.  Launched cooperatively, so every warp is
// resident; every phase reads only phases with a smaller index, warps take
// their phases in index order and pieces in list order, so the waits end.
template <typename T>
__global__ void __launch_bounds__(32 * kStreamWarps, 3) stream_kernel(const int4* __restrict__ recs, const __grid_constant__ GroupArgs<T> g,
                                                                   const __grid_constant__ Sched sc, typename V2<T>::t* __restrict__ P,
                                                                   int Pld, int* __restrict__ cnt, int* __restrict__ done,
                                                                   int* __restrict__ err)
{
    using C = typename V2<T>::t;
    using Cfg = StreamCfg<T>;
    extern __shared__ __align__(128) unsigned char smem[];
    // the leaf kernel after this launch may take SMs as CTAs retire; it waits
    // (griddepcontrol.wait) for this grid's writes before it reads them
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* wb = smem + (size_t)warp * Cfg::kWarp;
    auto stage = [&](int k) { return (C*)(wb + (size_t)k * Cfg::kStage); };
    C* xs = (C*)(wb + 2 * Cfg::kStage);
    unsigned long long* bar = (unsigned long long*)(wb + 2 * Cfg::kStage + Cfg::kXs);
    const int wg = warp * gridDim.x + blockIdx.x;  // the CTAs' first warps first
    {
        const int gt = wg * 32 + lane, nt = gridDim.x * kStreamWarps * 32;
        for (int r = 0; r < sc.npf; r++)
            for (long off = (long)gt * 128; off < sc.pf_bytes[r]; off += (long)nt * 128)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(sc.pf_ptr[r] + off));
    }
    unsigned long long pol;  // the operators are read once an application
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));

    // ---- scheduler (warp-uniform, except the lane-0 prefetches) ----
    Slice cs;
    bool hc = slice_from(sc, 0, wg, cs);  // a chain share is left
    bool in_share = false;                // scheduling inside the share cs
    int4 pc = make_int4(0, 0, 0, 0);      // piece being scheduled: {next chunk, end, slot, pass}
    int4 pq = make_int4(0, 0, 0, -1);     // lane 0: the next piece (pass -1: none left)
    int nid = 0;                          // lane 0: id of the piece after it
    unsigned ready = 0, seen = 0;         // passes known complete (acquired / polled)
    // A chain warp of its own (a share after phase 0) reserves no piece: a
    // reserved piece waits for its warp, and a chain warp may wait for the
    // pass that piece belongs to (an L2L reads the M2L of its level).
    Slice later;
    const bool takes_pieces = !(sc.chain_split && slice_from(sc, 1, wg, later));
    if (lane == 0 && sc.npieces > 0 && takes_pieces) {
        const int id0 = atomicAdd(sc.next_piece, 1);
        nid = atomicAdd(sc.next_piece, 1);
        if (id0 < sc.npieces) pq = sc.pieces[id0];
    }
    auto pick = [&]() {
        Item r;
        r.c = -1;
        r.kind = 0;
        r.aux = 0;
        r.end = 0;
        if (!in_share && pc.x >= pc.y) {
            const int4 e = shfl4(pq);
            const bool hb = e.w >= 0;
            if (!hc && !hb) return r;
            bool chain;
            if (!hc)
                chain = false;
            else if (!hb)
                chain = true;
            else if ((sc.phdeps[cs.k] & ~(ready | seen)) == 0)
                chain = true;
            else if ((sc.deps[e.w] & ~(ready | seen)) == 0)
                chain = false;
            else
                chain = !(sc.dphase[e.w] < cs.k - 1);
            if (chain) {
                in_share = true;
            } else {
                pc = e;
                if (lane == 0) {
                    pq = nid < sc.npieces ? sc.pieces[nid] : make_int4(0, 0, 0, -1);
                    nid = atomicAdd(sc.next_piece, 1);
                }
            }
        }
        if (in_share) {
            r.c = cs.c;
            r.kind = 0;
            r.aux = cs.k;
            r.end = cs.e;
            if (cs.c + 1 < cs.e) {
                cs.c++;
            } else {
                in_share = false;
                hc = slice_from(sc, cs.k + 1, wg, cs);
            }
        } else {
            r.c = pc.x;
            r.kind = 1;
            r.aux = pc.z;
            r.end = pc.y;
            pc.x++;
        }
        return r;
    };
    Item cur = pick();
    if (cur.c < 0) return;
    Item n1 = pick();
    Item n2 = n1.c >= 0 ? pick() : Item{-1, 0, 0, 0};
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        unsigned bytes;
        const char* src = chunk_src<T>(g, recs[2 * cur.c], recs[2 * cur.c + 1], bytes);
        tma_load(stage(0), src, bytes, &bar[0], pol);
        if (n1.c >= 0) {
            src = chunk_src<T>(g, recs[2 * n1.c], recs[2 * n1.c + 1], bytes);
            tma_load(stage(1), src, bytes, &bar[1], pol);
        }
    }
    __syncwarp();
    // records of the current and the next chunk, the next chunk's input
    // indices: loaded one chunk ahead, so that only the input values
    // themselves (used an iteration later) are in flight during a chunk
    int4 ra = recs[2 * cur.c], rb = recs[2 * cur.c + 1];
    int4 na = make_int4(-1, -1, 0, 0), nb = make_int4(0, 0, 0, 0);
    int xc[kMaxPrefetch], xi[kMaxPrefetch];  // input indices of the current and the next chunk
    gather_idx<T>(g, ra, lane, xc);
    if (n1.c >= 0) {
        na = recs[2 * n1.c];
        nb = recs[2 * n1.c + 1];
        gather_idx<T>(g, na, lane, xi);
    }
    bool have_x = false;
    C xr[kMaxPrefetch];
    Acc<T> acc;
    acc.zero();
    int pend_pass = 0, pend_n = 0;  // finished rows of one pass not yet counted (warp-uniform)
    auto publish = [&]() {
        if (pend_n) rows_done(done, pend_pass, pend_n, lane);
        pend_n = 0;
    };
    for (int it = 0;; it++) {
        const int s = it & 1;
        const unsigned parity = (unsigned)((it >> 1) & 1);
        const bool h1 = n1.c >= 0, h2 = n2.c >= 0;
        // a wait that gives up: flag it, let this warp's copies in flight land, leave
        auto bail = [&]() {
            if (lane == 0) {
                atomicExch(err, 1);
                mbar_wait(&bar[s], parity);
                if (h1) mbar_wait(&bar[s ^ 1], ((it + 1) >> 1) & 1);
            }
            __syncwarp();
        };
        if (!have_x) {
            // first chunk of a pass whose inputs were not yet known complete
            if (sc.deps[ra.x & 0xff] & ~ready) publish();
            if (deps_wait(sc, done, sc.deps[ra.x & 0xff], ready, lane) < 0) {
                bail();
                return;
            }
            gather_val<T>(g, ra, lane, xc, xr);
        }
        // readiness polls for the next choice (lane 0; consumed after this chunk)
        int q1 = -1, q2 = -1, v1 = 0, v2 = 0;
        if (lane == 0) {
            if (hc && !in_share) {
                const unsigned m = sc.phdeps[cs.k] & ~(ready | seen);
                if (m) {
                    q1 = __ffs(m) - 1;
                    v1 = ld_relaxed(&done[q1 * kDoneStride]);
                }
            }
            if (pc.x >= pc.y && pq.w >= 0) {
                const unsigned m = sc.deps[pq.w] & ~(ready | seen);
                if (m) {
                    q2 = __ffs(m) - 1;
                    v2 = ld_relaxed(&done[q2 * kDoneStride]);
                }
            }
        }
        // commit this chunk's inputs
        const int ncol = ra.z;
#pragma unroll
        for (int k = 0; k < kMaxPrefetch; k++) {
            const int t = lane + 32 * k;
            if (t < ncol) xs[t] = xr[k];
        }
        // records of the chunk after next; the next chunk's inputs when its passes are known complete
        int4 fa = make_int4(-1, -1, 0, 0), fb = make_int4(0, 0, 0, 0);
        if (h2) {
            fa = recs[2 * n2.c];
            fb = recs[2 * n2.c + 1];
        }
        have_x = false;
        if (h1 && (sc.deps[na.x & 0xff] & ~ready) == 0) {
            gather_val<T>(g, na, lane, xi, xr);
            have_x = true;
        }
        if (!__all_sync(0xffffffffu, mbar_wait(&bar[s], parity))) {
            bail();
            return;
        }
        __syncwarp();
        const int pass = ra.x & 0xff;
        const PassArgs<T>& pa = g.p[pass];
        const int ro = (ra.x >> 16) & 0xffff;
        const int ld = ro + (ro & 1);
        chunk_mac<T>(acc, stage(s), xs, ro, ld, ncol, lane);
        // every lane is done with this stage and the gather buffer: refill the stage
        __syncwarp();
        if (lane == 0 && h2) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            unsigned nbytes;
            const char* src = chunk_src<T>(g, fa, fb, nbytes);
            tma_load(stage(s), src, nbytes, &bar[s], pol);
        }
        if (!have_x) {
#pragma unroll
            for (int k = 0; k < kMaxPrefetch; k++) xc[k] = xi[k];  // the next chunk gathers at the top
        }
        if (h2) gather_idx<T>(g, fa, lane, xi);
        // end of this row's run in the unit: write it out
        const bool row_ends = !h1 || n1.kind != cur.kind || n1.aux != cur.aux || na.x != ra.x || na.y != ra.y;
        if (row_ends) {
            C* yrow = pa.y + (size_t)ra.y * pa.ldy;
            bool fin = true;
            if (cur.kind == 0) {
                const int b = sc.base[cur.aux] + (wg - sc.wlo[cur.aux]) * sc.kpw[cur.aux];
                if (rb.w < b) {
                    // the row began in an earlier share: leave a partial for its owner
                    flush_row<T>(acc, ro, lane, P + (size_t)share_slot(sc, cur.aux, b) * Pld, false, 0);
                    put_partial(cnt, rb.w, lane);
                    fin = false;
                } else {
                    flush_row<T>(acc, ro, lane, yrow, true, 0);
                    if (rb.z > cur.end) publish();
                    if (rb.z > cur.end && !own_row<T>(yrow, P, Pld, cnt, rb.w, rb.z, sc, cur.aux, ro, lane)) {
                        // the copies in flight now: the next chunk's (other stage), the one after (this stage)
                        if (lane == 0) {
                            atomicExch(err, 1);
                            if (h1) mbar_wait(&bar[s ^ 1], ((it + 1) >> 1) & 1);
                            if (h2) mbar_wait(&bar[s], ((it + 2) >> 1) & 1);
                        }
                        __syncwarp();
                        return;
                    }
                }
            } else if (rb.z - rb.w <= kPiece) {
                flush_row<T>(acc, ro, lane, yrow, true, 0);  // the piece is the whole row
            } else {
                flush_row<T>(acc, ro, lane, P + (size_t)cur.aux * Pld, false, 0);
                fin = bulk_finish<T>(yrow, P, Pld, cnt, rb.w, rb.z, cur.aux, cur.c, ro, lane);
            }
            if (fin && (sc.pub >> pass & 1u)) {
                if (pass != pend_pass) publish();
                pend_pass = pass;
                pend_n++;
            }
            acc.zero();
        }
        // the warp's run of the pass ends here: count its rows
        if (pend_n && (!h1 || (na.x & 0xff) != pend_pass)) publish();
        if (!h1) break;
        // fold in the polls, then choose the chunk after next
        unsigned add = 0;
        if (lane == 0) {
            if (q1 >= 0 && v1 >= sc.target[q1]) add |= 1u << q1;
            if (q2 >= 0 && v2 >= sc.target[q2]) add |= 1u << q2;
        }
        seen |= __shfl_sync(0xffffffffu, add, 0);
        const Item n3 = h2 ? pick() : Item{-1, 0, 0, 0};
        cur = n1;
        ra = na;
        rb = nb;
        n1 = n2;
        na = fa;
        nb = fb;
        n2 = n3;
    }
}

// ---------------------------------------------------------------------------
// Several right-hand sides (vectors [N][nrhs], coefficients [slot][R][nrhs]).
// One CTA streams a chunk range through the same TMA pipeline; its warps
// share each stage and split the right-hand sides (16 per warp).  Lane
// (r, g) of a warp owns right-hand side r and the contiguous rows
// [g h, g h + h) of the chunk's rows (h even, so rows come in 16-byte pairs
// for complex64); per column it reads its rows' entries from shared memory
// (broadcast across the 16 lanes of a half-warp) and the gathered input of
// its right-hand side.  The operator is read once for all right-hand sides.
constexpr int kRhsPerWarp = 16;
constexpr int kMaxChunkColsB = 32;  // columns of a chunk of the several-right-hand-side groups (input tile rows)

// A stage holds a chunk's matrix and its input tile [column][rhs] (row stride nrhs_pad).
template <typename T>
struct BatchCfg {
    using C = typename V2<T>::t;
    static constexpr int kMat = ((int)(kChunkElems * sizeof(C)) + 32 + 127) / 128 * 128;
    __host__ __device__ static int xs_bytes(int nrhs_pad) { return kMaxChunkColsB * nrhs_pad * (int)sizeof(C); }
    __host__ __device__ static int stage_bytes(int nrhs_pad) { return kMat + xs_bytes(nrhs_pad); }
    __host__ __device__ static int cta_bytes(int nrhs_pad) { return 2 * stage_bytes(nrhs_pad) + 128; }
};

// Start chunk c's copies into stage buffer st (matrix, then input tile) on
// barrier bar: thread 0 arms the barrier for every byte and copies the
// matrix; with bulk_x each input column (nrhs values, contiguous in x) is one
// bulk copy by thread k of the CTA, else the block gathers the inputs itself
// (synchronously, into the same tile).
template <typename T>
__device__ __forceinline__ void batch_issue(const GroupArgs<T>& g, const int4* recs, int c, unsigned char* st, unsigned long long* bar,
                                            int nrhs, int nrhs_pad, bool bulk_x, int tid, int nthr)
{
    using C = typename V2<T>::t;
    const int4 a = recs[2 * c], b = recs[2 * c + 1];
    const PassArgs<T>& pa = g.p[a.x & 0xff];
    const int ncol = a.z;
    const unsigned xbytes = (unsigned)(nrhs * sizeof(C));
    C* xt = (C*)(st + BatchCfg<T>::kMat);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0) {
        unsigned mbytes;
        const char* src = chunk_src<T>(g, a, b, mbytes);
        const unsigned total = mbytes + (bulk_x ? (unsigned)ncol * xbytes : 0u);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(total) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(st)),
                     "l"(src), "r"(mbytes), "r"(smem_u32(bar))
                     : "memory");
    }
    if (bulk_x) {
        for (int k = tid; k < ncol; k += nthr) {
            const C* src = pa.x + (size_t)pa.xmap[a.w + k] * nrhs;
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             smem_u32(xt + (size_t)k * nrhs_pad)),
                         "l"(src), "r"(xbytes), "r"(smem_u32(bar))
                         : "memory");
        }
    }
}

// acc[m] += M[m][k] x[k] over the chunk's columns for H rows of one lane (H
// even, rows [i0, i0 + H) of a column of ld entries at M; x[k] at xs[k xst]).
// Rows past the chunk's row count compute values that are never stored; their
// reads stay inside the stage (the matrix is at most ld x ncol <= 1024 entries
// and at most two rows past the last column are read, into the stage slack).
// Columns are unrolled by U so that a lane with few rows still has about 16
// independent products in flight between shared-memory loads.
template <int H, int MR>
__device__ __forceinline__ void batch_rows_h(float (&ar)[MR], float (&ai)[MR], const float2* M, const float2* xs, int ncol, int ld, int xst)
{
    constexpr int U = H >= 16 ? 1 : 16 / H;
    int k = 0;
    for (; k + U <= ncol; k += U) {
        float2 xv[U];
        float4 mm[U][H / 2];
#pragma unroll
        for (int u = 0; u < U; u++) {
            xv[u] = xs[(k + u) * xst];
#pragma unroll
            for (int m = 0; m < H / 2; m++) mm[u][m] = *(const float4*)(M + (k + u) * ld + 2 * m);
        }
#pragma unroll
        for (int u = 0; u < U; u++)
#pragma unroll
            for (int m = 0; m < H / 2; m++) {
                const float4 q = mm[u][m];
                const float2 x = xv[u];
                ar[2 * m] = fmaf(q.x, x.x, fmaf(-q.y, x.y, ar[2 * m]));
                ai[2 * m] = fmaf(q.x, x.y, fmaf(q.y, x.x, ai[2 * m]));
                ar[2 * m + 1] = fmaf(q.z, x.x, fmaf(-q.w, x.y, ar[2 * m + 1]));
                ai[2 * m + 1] = fmaf(q.z, x.y, fmaf(q.w, x.x, ai[2 * m + 1]));
            }
    }
    for (; k < ncol; k++) {
        const float2 x = xs[k * xst];
#pragma unroll
        for (int m = 0; m < H / 2; m++) {
            const float4 q = *(const float4*)(M + k * ld + 2 * m);
            ar[2 * m] = fmaf(q.x, x.x, fmaf(-q.y, x.y, ar[2 * m]));
            ai[2 * m] = fmaf(q.x, x.y, fmaf(q.y, x.x, ai[2 * m]));
            ar[2 * m + 1] = fmaf(q.z, x.x, fmaf(-q.w, x.y, ar[2 * m + 1]));
            ai[2 * m + 1] = fmaf(q.z, x.y, fmaf(q.w, x.x, ai[2 * m + 1]));
        }
    }
}

// Complex128 (float pairs, double-float arithmetic as in Acc<double>):
// acc[m] += M[m][k] x[k] with (hi, lo) accumulators per row.
template <int H, int MR>
__device__ __forceinline__ void batch_rows_df_h(float (&rh)[MR], float (&rl)[MR], float (&ih)[MR], float (&il)[MR], const double2* M,
                                                const double2* xs, int ncol, int ld, int xst)
{
    for (int k = 0; k < ncol; k++) {
        const float4 x = as_df(xs[k * xst]);
#pragma unroll
        for (int m = 0; m < H; m++) df_cmac(rh[m], rl[m], ih[m], il[m], as_df(M[k * ld + m]), x);
    }
}

template <int MR, int H = 2>
__device__ __forceinline__ void batch_rows_df(int h, float (&rh)[MR], float (&rl)[MR], float (&ih)[MR], float (&il)[MR], const double2* M,
                                              const double2* xs, int ncol, int ld, int xst)
{
    if constexpr (H <= MR) {
        if (h == H)
            batch_rows_df_h<H, MR>(rh, rl, ih, il, M, xs, ncol, ld, xst);
        else
            batch_rows_df<MR, H + 2>(h, rh, rl, ih, il, M, xs, ncol, ld, xst);
    }
}

// Dispatch on the lane's row count h (even, at most MR; uniform over the CTA).
template <int MR, int H = 2>
__device__ __forceinline__ void batch_rows(int h, float (&ar)[MR], float (&ai)[MR], const float2* M, const float2* xs, int ncol, int ld,
                                           int xst)
{
    if constexpr (H <= MR) {
        if (h == H)
            batch_rows_h<H, MR>(ar, ai, M, xs, ncol, ld, xst);
        else
            batch_rows<MR, H + 2>(h, ar, ai, M, xs, ncol, ld, xst);
    }
}

template <typename T, int MR>
__global__ void __launch_bounds__(128) stream_batched_kernel(int nch, int kpc, int nrhs, int nrhs_pad, int bulk_x, const int4* __restrict__ recs,
                                                             const __grid_constant__ GroupArgs<T> g,
                                                             typename V2<T>::t* __restrict__ P, int Pld, int* __restrict__ cnt,
                                                             int* __restrict__ err)
{
    using C = typename V2<T>::t;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sb = BatchCfg<T>::stage_bytes(nrhs_pad);
    auto stage_raw = [&](int k) { return smem + (size_t)k * sb; };
    auto stage = [&](int k) { return (C*)stage_raw(k); };
    auto tile = [&](int k) { return (C*)(stage_raw(k) + BatchCfg<T>::kMat); };
    unsigned long long* bar = (unsigned long long*)(smem + 2 * (size_t)sb);
    const int r = warp * kRhsPerWarp + (lane & 15);
    const int gsel = lane >> 4;
    const int cb = blockIdx.x * kpc;
    const int ce = min(nch, cb + kpc);
    if (cb >= ce) return;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    for (int k = 0; k < 2 && cb + k < ce; k++) batch_issue<T>(g, recs, cb + k, stage_raw(k), &bar[k], nrhs, nrhs_pad, bulk_x, tid, blockDim.x);
    // complex64: FP32 accumulators; complex128: float pairs (double-float)
    float ar[MR], ai[MR], al[MR], bl[MR];
#pragma unroll
    for (int m = 0; m < MR; m++) ar[m] = ai[m] = al[m] = bl[m] = 0.f;
    int pslot = cb;
    for (int c = cb, it = 0; c < ce; c++, it++) {
        const int s = it & 1;
        const unsigned parity = (unsigned)((it >> 1) & 1);
        const int4 ra = recs[2 * c];
        const PassArgs<T>& pa = g.p[ra.x & 0xff];
        const int ro = (ra.x >> 16) & 0xffff;
        const int ld = ro + (ro & 1);
        const int ncol = ra.z;
        C* xs = tile(s);
        if (!bulk_x) {
            // gather this chunk's inputs for every right-hand side: xs[k][rr]
            for (int q = tid; q < ncol * nrhs; q += blockDim.x) {
                const int k = q / nrhs, rr = q - k * nrhs;
                xs[k * nrhs_pad + rr] = pa.x[(size_t)pa.xmap[ra.w + k] * nrhs + rr];
            }
        }
        const bool ok = __syncthreads_and(mbar_wait(&bar[s], parity));
        if (!ok) {
            if (tid == 0) {
                atomicExch(err, 1);
                mbar_wait(&bar[s], parity);
                if (c + 1 < ce) mbar_wait(&bar[s ^ 1], ((it + 1) >> 1) & 1);
            }
            __syncthreads();
            return;
        }
        // rows of this lane: [gsel h, gsel h + h), h even
        const int h = ((ro + 3) >> 2) << 1;
        const int i0 = gsel * h;
        if (r < nrhs) {
            if constexpr (sizeof(T) == 8)
                batch_rows_df<MR>(h, ar, al, ai, bl, stage(s) + i0, xs + r, ncol, ld, nrhs_pad);
            else
                batch_rows<MR>(h, ar, ai, stage(s) + i0, xs + r, ncol, ld, nrhs_pad);
        }
        __syncthreads();  // everyone is done with this stage (matrix and inputs)
        if (c + 2 < ce) batch_issue<T>(g, recs, c + 2, stage_raw(s), &bar[s], nrhs, nrhs_pad, bulk_x, tid, blockDim.x);
        const bool row_ends = (c + 1 == ce) || recs[2 * (c + 1)].x != ra.x || recs[2 * (c + 1)].y != ra.y;
        if (row_ends) {
            const bool direct = (ra.x & kFlagDirect) != 0;
            const bool add = (ra.x & kFlagAdd) != 0;
            C* yrow = pa.y + (size_t)ra.y * pa.ldy * nrhs;
            const int4 rbx = recs[2 * c + 1];
            const bool whole = direct || (rbx.w >= cb && rbx.z <= ce);  // every chunk of the row is in this CTA's range
            if (r < nrhs) {
                C* dst = whole ? yrow : P + (size_t)pslot * Pld * nrhs;
#pragma unroll
                for (int m = 0; m < MR; m++) {
                    const int i = i0 + m;
                    if (i < ro && m < h) {
                        C* q = dst + (size_t)i * nrhs + r;
                        if constexpr (sizeof(T) == 8) {
                            float4 o = make_float4(ar[m], ai[m], al[m], bl[m]);
                            if (whole && add) o = df4_add(o, as_df(*q));
                            *q = df_bits(o);
                        } else {
                            T re = ar[m], im = ai[m];
                            if (whole && add) {
                                const C o = *q;
                                re += o.x;
                                im += o.y;
                            }
                            C o;
                            o.x = re;
                            o.y = im;
                            *q = o;
                        }
                    }
                    ar[m] = ai[m] = al[m] = bl[m] = 0.f;
                }
            }
            if (!whole) {
                // the last CTA to write a partial of this row sums them in slot order
                const int c0 = rbx.w, c1 = rbx.z;
                __threadfence();
                __syncthreads();
                if (tid == 0) s_last = atomicAdd(&cnt[c0], 1) + 1 == row_slots(c0, c1, 0, kpc);
                __syncthreads();
                if (s_last) {
                    __threadfence();
                    for (int qq = tid; qq < ro * nrhs; qq += blockDim.x) {
                        if constexpr (sizeof(T) == 8) {
                            float4 acc = add ? as_df(yrow[qq]) : make_float4(0.f, 0.f, 0.f, 0.f);
                            for (int cc = c0; cc < c1; cc = (cc / kpc + 1) * kpc)
                                acc = df4_add(acc, as_df(__ldcg(&P[(size_t)cc * Pld * nrhs + qq])));
                            yrow[qq] = df_bits(acc);
                        } else {
                            T sr = 0, si = 0;
                            if (add) {
                                const C o = yrow[qq];
                                sr = o.x;
                                si = o.y;
                            }
                            for (int cc = c0; cc < c1; cc = (cc / kpc + 1) * kpc) {
                                const C p = __ldcg(&P[(size_t)cc * Pld * nrhs + qq]);
                                sr += p.x;
                                si += p.y;
                            }
                            C o;
                            o.x = sr;
                            o.y = si;
                            yrow[qq] = o;
                        }
                    }
                    if (tid == 0) cnt[c0] = 0;
                }
                __syncthreads();
            }
            pslot = c + 1;
        }
    }
}

// ---------------------------------------------------------------------------
// Several right-hand sides on the tensor cores (complex64 operators).  A
// chunk's product Y[i][r] += sum_k M[i][k] X[k][r] (i < ro rows, k < ncol
// columns, r < nrhs <= 64) is a real GEMM after the usual embedding of
// complex numbers: with a K index 2k + t (t = 0 real part, 1 imaginary part
// of X[k][r]) the 2 NR output columns are [Re Y_0 .. Re Y_{ro-1} | pad |
// Im Y_0 ..] and B[i][2k] = Re M, B[i][2k+1] = -Im M, B[NR+i][2k] = Im M,
// B[NR+i][2k+1] = Re M.  tcgen05.mma kind::tf32 (D in TMEM, FP32) multiplies
// 11-bit significands, so every FP32 value v is split exactly into three
// tf32 parts v = h + m + l (h = rn(v), m = rn(v - h), l = v - h - m).  A
// holds X_h in rows 0..63 and X_m in rows 64..127 (M = 128) and A2 holds X_l
// over zeros; per K step D += A B_h + A B_m + A B_l + A2 B_h, so D rows r and
// 64 + r together hold every partial product down to 2^-33 relative (terms
// below are dropped), i.e. the FP32 products of the CUDA-core kernel.  The
// tensor core's own FP32 accumulation over a long chain of MMAs loses more
// than rounded FMAs do (measured: five times the CUDA-core kernel's error
// when a row's whole chain accumulated in TMEM), so each chunk's MMAs start a
// fresh accumulator (at most 32 MMAs deep) that is drained into FP32
// registers with rounded additions (tcgen05.ld) before the next chunk's
// MMAs.  Operands are K-major 8 x 16-byte core matrices without swizzle.
constexpr int kTcThreads = 256;
constexpr int kTcRaw = 3;              // bulk-copy stages of raw chunks
constexpr int kTcA = 128 * 64 * 4;     // A (and A2) operand: 128 rows x 64 K (tf32)
constexpr int kTcBPart = 5120 * 4;     // one tf32 part of B for the largest chunk shape (2 NR x Kpad <= 5120)
constexpr int kTcB = 3 * kTcBPart;
constexpr int kTcCols = 128;           // TMEM columns (N = 2 NR <= 128)
constexpr int kTcIssuer = kTcThreads - 32;  // the thread that issues and commits the MMAs (lane 0 of the last warp)

__host__ __device__ inline int tc_raw_bytes(int nrhs_pad) { return BatchCfg<float>::stage_bytes(nrhs_pad); }
__host__ __device__ inline int tc_smem_bytes(int nrhs_pad) { return kTcRaw * tc_raw_bytes(nrhs_pad) + 2 * kTcA + kTcB + 128; }

// Byte offset of element (row, k) of a K-major operand with Kt columns: core
// matrix (row / 8, k / 4) at 128 bytes each, row-group major.
__device__ __forceinline__ unsigned tc_off(int row, int k, int Kt)
{
    return (unsigned)((((row >> 3) * (Kt >> 2) + (k >> 2)) << 7) + ((row & 7) << 4) + ((k & 3) << 2));
}

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (between core matrices along K), stride byte offset (between
// 8-row groups), descriptor version 1, no swizzle.
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr, unsigned lbo, unsigned sbo)
{
    return (unsigned long long)((addr >> 4) & 0x3FFF) | ((unsigned long long)((lbo >> 4) & 0x3FFF) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ float tc_rn(float v)
{
    unsigned h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
    return __uint_as_float(h);
}

// v = h + m + l exactly, each a tf32 value.
__device__ __forceinline__ void tc_split3(float v, float& h, float& m, float& l)
{
    h = tc_rn(v);
    const float r = v - h;  // exact
    m = tc_rn(r);
    l = tc_rn(r - m);       // exact: at most two significant bits remain
}

// Chunk in raw stage (matrix M, ld x ncol column-major; inputs xs[k][r]) ->
// operands A, A2 (128 x Kpad) and the three parts of B (N x Kpad).  Rows of B
// past ro and rows of A, A2 past nrhs only reach accumulator rows or columns
// the epilogue never reads, except the rows 64..64+nrhs of A2, which are
// zeroed.  The K padding is zero in every operand.
__device__ __forceinline__ void tc_convert(const float2* M, int ld, int ro, int NR, int ncol, int Kpad, const float2* xs, int nrhs_pad,
                                           int nrhs, unsigned char* A, unsigned char* A2, unsigned char* B, int tid)
{
    for (int e = tid; e < ro * ncol; e += kTcThreads) {
        const int k = e / ro, i = e - k * ro;
        const float2 mv = M[k * ld + i];
        float r[3], im[3];
        tc_split3(mv.x, r[0], r[1], r[2]);
        tc_split3(mv.y, im[0], im[1], im[2]);
        const unsigned o1 = tc_off(i, 2 * k, Kpad), o2 = tc_off(NR + i, 2 * k, Kpad);
#pragma unroll
        for (int p = 0; p < 3; p++) {
            *(float2*)(B + p * kTcBPart + o1) = make_float2(r[p], -im[p]);
            *(float2*)(B + p * kTcBPart + o2) = make_float2(im[p], r[p]);
        }
    }
    for (int e = tid; e < ncol * 64; e += kTcThreads) {
        const int k = e >> 6, r = e & 63;
        if (r < nrhs) {
            const float2 x = xs[k * nrhs_pad + r];
            float a[3], b[3];
            tc_split3(x.x, a[0], a[1], a[2]);
            tc_split3(x.y, b[0], b[1], b[2]);
            *(float2*)(A + tc_off(r, 2 * k, Kpad)) = make_float2(a[0], b[0]);
            *(float2*)(A + tc_off(64 + r, 2 * k, Kpad)) = make_float2(a[1], b[1]);
            *(float2*)(A2 + tc_off(r, 2 * k, Kpad)) = make_float2(a[2], b[2]);
            *(float2*)(A2 + tc_off(64 + r, 2 * k, Kpad)) = make_float2(0.f, 0.f);
        }
    }
    const int kp = Kpad - 2 * ncol;  // zero K padding (0, 2, 4 or 6 columns)
    if (kp > 0) {
        const int N = 2 * NR;
        for (int e = tid; e < (128 + N) * kp; e += kTcThreads) {
            const int row = e / kp, k = 2 * ncol + (e - row * kp);
            if (row < 128) {
                *(float*)(A + tc_off(row, k, Kpad)) = 0.f;
                *(float*)(A2 + tc_off(row, k, Kpad)) = 0.f;
            } else {
#pragma unroll
                for (int p = 0; p < 3; p++) *(float*)(B + p * kTcBPart + tc_off(row - 128, k, Kpad)) = 0.f;
            }
        }
    }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// One tcgen05.mma (kind::tf32, one CTA): D (+)= A B^T with the given descriptors.
__device__ __forceinline__ void tc_mma(unsigned tmem, unsigned long long ad, unsigned long long bd, unsigned idesc, unsigned acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                 "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                 : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned long long* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 8 consecutive accumulator columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tc_ld8(unsigned taddr, float (&v)[8])
{
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 8; j++) v[j] = __uint_as_float(r[j]);
}

// The several-right-hand-side pass on the tensor cores: the chunk ranges and
// split-row handling of stream_batched_kernel with a three-stage bulk-copy
// pipeline of raw chunks.  Per chunk: wait for its raw stage and for the
// previous chunk's MMAs (one operand set), convert, one thread issues the
// MMAs and commits them to the MMA barrier; at the end of a row the
// accumulator goes through shared memory to the row's output.  Every wait is
// bounded; on a timeout the CTA raises the device flag, waits (bounded) for
// its copies and MMAs, frees its TMEM and returns.
__global__ void __launch_bounds__(kTcThreads, 1) stream_batched_tc_kernel(int nch, int kpc, int nrhs, int nrhs_pad, int bulk_x,
                                                                          const int4* __restrict__ recs,
                                                                          const __grid_constant__ GroupArgs<float> g, float2* __restrict__ P,
                                                                          int Pld, int* __restrict__ cnt, int* __restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_last;
    __shared__ int s_bad;
    __shared__ unsigned s_tmem;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cb = blockIdx.x * kpc;
    const int ce = min(nch, cb + kpc);
    if (cb >= ce) return;
    const int rb = tc_raw_bytes(nrhs_pad);
    auto raw = [&](int k) { return smem + k * rb; };
    unsigned char* A = smem + kTcRaw * rb;
    unsigned char* A2 = A + kTcA;
    unsigned char* B = A2 + kTcA;
    float* E = (float*)A;  // epilogue: accumulator columns x 128 lanes (overlays A and A2)
    unsigned long long* bar = (unsigned long long*)(B + kTcB);  // [0, kTcRaw) raw stages, [kTcRaw] MMAs
    unsigned long long* mbar = bar + kTcRaw;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)), "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int k = 0; k <= kTcRaw; k++) mbar_init(&bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_bad = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = s_tmem;
    int pend[kTcRaw];  // per raw stage: parity of a copy issued and not yet waited for
#pragma unroll
    for (int k = 0; k < kTcRaw; k++) {
        pend[k] = -1;
        if (cb + k < ce) {
            if (warp == 0) batch_issue<float>(g, recs, cb + k, raw(k), &bar[k], nrhs, nrhs_pad, bulk_x, lane, 32);
            pend[k] = 0;
        }
    }
    int pslot = cb;
    int issued = 0;        // chunks whose MMAs were committed
    bool undrained = false;  // the previous chunk's accumulator is still in TMEM
    int prevN = 0;           // its column count
    // this thread's share of the row's accumulator: TMEM lane 32 (warp & 3) +
    // lane, columns (warp >> 2) N/2 + j
    float acc[64];
#pragma unroll
    for (int j = 0; j < 64; j++) acc[j] = 0.f;
    auto drain = [&](int N) {
        const int q = warp & 3, half = N >> 1, col0 = (warp >> 2) * half;
#pragma unroll
        for (int g8 = 0; g8 < 8; g8++)
            if (8 * g8 < half) {
                float v[8];
                tc_ld8(tmem + ((unsigned)(32 * q) << 16) + (unsigned)(col0 + 8 * g8), v);
#pragma unroll
                for (int j = 0; j < 8; j++) acc[8 * g8 + j] += v[j];
            }
    };
    int4 na = recs[2 * cb];  // the next chunk's record, loaded a chunk ahead
    for (int c = cb, it = 0; c < ce; c++, it++) {
        const int s = it % kTcRaw;
        const int4 ra = na;
        if (c + 1 < ce) na = recs[2 * (c + 1)];
        const PassArgs<float>& pa = g.p[ra.x & 0xff];
        const int ro = (ra.x >> 16) & 0xffff;
        const int ld = ro + (ro & 1);
        const int ncol = ra.z;
        const int NR = (ro + 7) & ~7;
        const int Kpad = 2 * ((ncol + 3) & ~3);
        float2* xs = (float2*)(raw(s) + BatchCfg<float>::kMat);
        if (!bulk_x)
            for (int q = tid; q < ncol * nrhs; q += kTcThreads) {
                const int k = q / nrhs, rr = q - k * nrhs;
                xs[k * nrhs_pad + rr] = pa.x[(size_t)pa.xmap[ra.w + k] * nrhs + rr];
            }
        bool ok = mbar_wait(&bar[s], (unsigned)((it / kTcRaw) & 1));  // raw stage arrived
        if (ok) pend[s] = -1;
        if (it >= 1) ok = ok && mbar_wait(mbar, (unsigned)((it - 1) & 1));  // the operands are free
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicExch(err, 1);
            s_bad = 1;
            break;
        }
        tc_fence_after();
        if (undrained) drain(prevN);  // the previous chunk's MMAs are complete
        tc_convert((const float2*)raw(s), ld, ro, NR, ncol, Kpad, xs, nrhs_pad, nrhs, A, A2, B, tid);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();  // operands written; the raw stage is free again
        // warp 0 issues the bulk copies of the chunk kTcRaw ahead (their addresses need
        // global loads) while a lane of the last warp issues this chunk's MMAs
        if (c + kTcRaw < ce) {
            if (warp == 0) batch_issue<float>(g, recs, c + kTcRaw, raw(s), &bar[s], nrhs, nrhs_pad, bulk_x, lane, 32);
            pend[s] = ((it + kTcRaw) / kTcRaw) & 1;
        }
        if (tid == kTcIssuer) {
            tc_fence_after();
            const int N = 2 * NR;
            const unsigned idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(128 >> 4) << 24);
            const unsigned sbo = (unsigned)(Kpad >> 2) << 7;
            const unsigned a0 = smem_u32(A), a20 = smem_u32(A2), b0 = smem_u32(B);
            for (int st = 0; st < Kpad / 8; st++) {
                const unsigned long long ad = tc_desc(a0 + 256 * st, 128, sbo);
                const unsigned long long bh = tc_desc(b0 + 256 * st, 128, sbo);
                tc_mma(tmem, ad, bh, idesc, st == 0 ? 0u : 1u);
                tc_mma(tmem, ad, tc_desc(b0 + kTcBPart + 256 * st, 128, sbo), idesc, 1u);
                tc_mma(tmem, ad, tc_desc(b0 + 2 * kTcBPart + 256 * st, 128, sbo), idesc, 1u);
                tc_mma(tmem, tc_desc(a20 + 256 * st, 128, sbo), bh, idesc, 1u);
            }
            tc_commit(mbar);
        }
        issued = it + 1;
        undrained = true;
        prevN = 2 * NR;
        const bool row_ends = (c + 1 == ce) || na.x != ra.x || na.y != ra.y;
        if (!row_ends) continue;
        // the row's accumulator: wait for its last MMAs, drain, columns to E[n][lane]
        ok = mbar_wait(mbar, (unsigned)(it & 1));
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicExch(err, 1);
            s_bad = 1;
            break;
        }
        tc_fence_after();
        drain(prevN);
        undrained = false;
        {
            const int q = warp & 3, half = NR, col0 = (warp >> 2) * half;
#pragma unroll
            for (int j = 0; j < 64; j++)
                if (j < half) {
                    E[(col0 + j) * 128 + 32 * q + lane] = acc[j];
                    acc[j] = 0.f;
                }
        }
        tc_fence_before();
        __syncthreads();
        const bool direct = (ra.x & kFlagDirect) != 0;
        const bool add = (ra.x & kFlagAdd) != 0;
        float2* yrow = pa.y + (size_t)ra.y * pa.ldy * nrhs;
        const int4 rbx = recs[2 * c + 1];
        const bool whole = direct || (rbx.w >= cb && rbx.z <= ce);
        float2* dst = whole ? yrow : P + (size_t)pslot * Pld * nrhs;
        for (int e = tid; e < ro * nrhs; e += kTcThreads) {
            const int i = e / nrhs, r = e - i * nrhs;
            float re = E[i * 128 + r] + E[i * 128 + 64 + r];
            float im = E[(NR + i) * 128 + r] + E[(NR + i) * 128 + 64 + r];
            float2* qp = dst + (size_t)i * nrhs + r;
            if (whole && add) {
                const float2 o = *qp;
                re += o.x;
                im += o.y;
            }
            *qp = make_float2(re, im);
        }
        if (!whole) {
            // the last CTA to write a partial of this row sums them in slot order
            const int c0 = rbx.w, c1 = rbx.z;
            __threadfence();
            __syncthreads();
            if (tid == 0) s_last = atomicAdd(&cnt[c0], 1) + 1 == row_slots(c0, c1, 0, kpc);
            __syncthreads();
            if (s_last) {
                __threadfence();
                for (int qq = tid; qq < ro * nrhs; qq += kTcThreads) {
                    float sr = 0, si = 0;
                    if (add) {
                        const float2 o = yrow[qq];
                        sr = o.x;
                        si = o.y;
                    }
                    for (int cc = c0; cc < c1; cc = (cc / kpc + 1) * kpc) {
                        const float2 p = __ldcg(&P[(size_t)cc * Pld * nrhs + qq]);
                        sr += p.x;
                        si += p.y;
                    }
                    yrow[qq] = make_float2(sr, si);
                }
                if (tid == 0) cnt[c0] = 0;
            }
        }
        __syncthreads();  // E (the A operands) is free for the next conversion
        pslot = c + 1;
    }
    if (s_bad && tid == 0) {
        // let this CTA's copies and MMAs in flight land (bounded) before the TMEM goes
        for (int k = 0; k < kTcRaw; k++)
            if (pend[k] >= 0) mbar_wait(&bar[k], (unsigned)pend[k]);
    }
    if (s_bad && tid == kTcIssuer && issued > 0) mbar_wait(mbar, (unsigned)((issued - 1) & 1));
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
}

// Batched leaf kernel: one CTA per leaf, threads over (node i, rhs r), rhs fastest.
template <typename T>
__global__ void leaf_batched_kernel(int nleaf, int nrhs, const int* __restrict__ nbr, const typename V2<T>::t* __restrict__ near,
                                    const typename V2<T>::t* __restrict__ vin, const int* __restrict__ l2p_rowptr,
                                    const long* __restrict__ l2p_moff, const int* __restrict__ l2p_rin,
                                    const typename V2<T>::t* __restrict__ l2p, int ldl, const typename V2<T>::t* __restrict__ lc,
                                    const double2* __restrict__ v, const double* __restrict__ q, double k2, double2* __restrict__ out)
{
    using C = typename V2<T>::t;
    __shared__ C sn[9 * 256];
    for (int k = threadIdx.x; k < 9 * 256; k += blockDim.x) sn[k] = near[k];
    __syncthreads();
    const int leaf = blockIdx.x;
    for (int t = threadIdx.x; t < 16 * nrhs; t += blockDim.x) {
        const int i = t / nrhs, r = t - i * nrhs;
        T ar = 0, ai = 0;
        // complex128: near blocks, inputs, L2P and locals are float pairs (double-float)
        float dh = 0.f, dl = 0.f, eh = 0.f, el = 0.f;
        for (int o = 0; o < 9; o++) {
            const int src = nbr[leaf * 9 + o];
            if (src < 0) continue;
            const C* vs = vin + (size_t)src * 16 * nrhs + r;
            const C* B = sn + o * 256 + i;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                if constexpr (sizeof(T) == 8)
                    df_cmac(dh, dl, eh, el, as_df(B[j * 16]), as_df(vs[(size_t)j * nrhs]));
                else
                    cmac<T>(ar, ai, B[j * 16], vs[(size_t)j * nrhs]);
            }
        }
        if (l2p_rowptr != nullptr && l2p_rowptr[leaf + 1] > l2p_rowptr[leaf]) {
            const int e = l2p_rowptr[leaf];
            const C* U = l2p + l2p_moff[e] + i;
            const C* u = lc + (size_t)leaf * ldl * nrhs + r;
            const int ri = l2p_rin[e];
            for (int j = 0; j < ri; j++) {
                if constexpr (sizeof(T) == 8)
                    df_cmac(dh, dl, eh, el, as_df(U[j * 16]), as_df(u[(size_t)j * nrhs]));
                else
                    cmac<T>(ar, ai, U[j * 16], u[(size_t)j * nrhs]);
            }
        }
        if constexpr (sizeof(T) == 8) {
            ar = (double)dh + (double)dl;
            ai = (double)eh + (double)el;
        }
        const size_t gi = ((size_t)leaf * 16 + i) * nrhs + r;
        if (q == nullptr) {
            out[gi] = make_double2((double)ar, (double)ai);  // the potential K v alone
        } else {
            const double2 vv = v[gi];
            const double sc = k2 * q[(size_t)leaf * 16 + i];
            out[gi] = make_double2(vv.x + sc * (double)ar, vv.y + sc * (double)ai);
        }
    }
}

// out = v + kappa^2 q (U_B u^{B,i} + sum_{9 offsets} T_o v_{B+o}) per leaf.
// 48 threads per leaf: node i and one row sy of the 3 x 3 near offsets each;
// the first group stages shared memory, every group applies its row of near
// offsets, and after the wait for the launch before (griddepcontrol) the
// second applies the composed L2L and L2P and the third L2P; the groups'
// sums meet in shared memory.
// 4 leaves per CTA.  Near blocks are stored [o][j][i] (target index fastest)
// for conflict-free shared reads.  A CTA's four leaves are consecutive in
// Morton order (a 2 x 2 quad); the inputs of the 4 x 4 leaves around it are
// read in complex128, rounded to T once and kept in shared memory (FP64
// conversions are scarce on this GPU).  The leaves' locals are lc (+ lc2 when
// not null).  c_* (not null): blocks of the L2L from the parent level composed
// with L2P (16 x ri, column stride 16) applied by the second thread group to
// the parent level's locals lcA (+ lcB when not null), stride ldc.  done (not
// null): row and piece counters of the fused launch before, reset here for
// the next application.
constexpr int kLeafPerCta = 4;
constexpr int kLeafEnt = 8;        // composed blocks a leaf at most, for the staged far field
constexpr int kLeafStageCols = 64; // staged columns a leaf at most, composed and L2P each

// Bulk copies counted on an mbarrier: the expected bytes first, then the
// copy (both addresses 16-byte aligned, bytes a multiple of 16, pieces of
// at most 16 KB); each issuing thread arrives once when it has issued all.
__device__ __forceinline__ void bulk_expect_copy(void* dst, const void* src, unsigned bytes, unsigned long long* bar)
{
    for (unsigned o = 0; o < bytes; o += 16384) {
        const unsigned n = min(16384u, bytes - o);
        asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(n) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32((char*)dst + o)),
                     "l"((const char*)src + o), "r"(n), "r"(smem_u32(bar))
                     : "memory");
    }
}
__device__ __forceinline__ void mbar_arrive1(unsigned long long* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <typename T>
__global__ void __launch_bounds__(48 * kLeafPerCta) leaf_apply_kernel(int nleaf, const int* __restrict__ nbr,
                                                                      const typename V2<T>::t* __restrict__ near,
                                                                      const int* __restrict__ l2p_rowptr, const long* __restrict__ l2p_moff,
                                                                      const int* __restrict__ l2p_rin,
                                                                      const typename V2<T>::t* __restrict__ l2p, int ldl,
                                                                      const typename V2<T>::t* __restrict__ lc,
                                                                      const typename V2<T>::t* __restrict__ lc2,
                                                                      const int* __restrict__ c_rowptr, const int* __restrict__ c_col,
                                                                      const long* __restrict__ c_moff, const int* __restrict__ c_rin,
                                                                      const typename V2<T>::t* __restrict__ cm, int ldc,
                                                                      const typename V2<T>::t* __restrict__ lcA,
                                                                      const typename V2<T>::t* __restrict__ lcB,
                                                                      const double2* __restrict__ v, const double* __restrict__ q, double k2,
                                                                      double2* __restrict__ out, int* __restrict__ done, int fcc, int fcl,
                                                                      int* __restrict__ err)
{
    using C = typename V2<T>::t;
    static_assert(kLeafPerCta == 4, "a CTA takes one 2 x 2 quad of leaves (four consecutive Morton indices)");
    // fcc, fcl > 0: the far-field blocks are staged in shared memory, up to
    // fcc composed and fcl L2P columns a leaf: sUc [leaf][col][16], sUl the
    // same, then the locals they multiply, suc [leaf][col] and sul
    extern __shared__ __align__(16) unsigned char leaf_dyn[];
    const bool staged = fcc > 0 || fcl > 0;
    C* sUc = (C*)leaf_dyn;
    C* sUl = sUc + kLeafPerCta * fcc * 16;
    C* suc = sUl + kLeafPerCta * fcl * 16;
    C* sul = suc + kLeafPerCta * fcc;
    __shared__ int s_ecol[kLeafPerCta][kLeafEnt], s_erin[kLeafPerCta][kLeafEnt], s_ecoff[kLeafPerCta][kLeafEnt];
    __shared__ int s_nce[kLeafPerCta], s_ncc[kLeafPerCta], s_nl[kLeafPerCta];
    __shared__ __align__(16) C sn[9 * 256];
    __shared__ __align__(16) C vq[16][16];  // inputs of the 4 x 4 leaves around the quad, rounded to T once
                                            // (complex128: split into float pairs, like sn)
    __shared__ C part[2][kLeafPerCta * 16];
    auto rnd = [](double2 d) {
        C c;
        c.x = (T)d.x;
        c.y = (T)d.y;
        return c;
    };
    const int q0 = blockIdx.x * kLeafPerCta;
    const int grp = threadIdx.x / (16 * kLeafPerCta);  // offset row sy = grp - 1 of the near field
    const int li = threadIdx.x % (16 * kLeafPerCta);
    const int leaf = blockIdx.x * kLeafPerCta + li / 16;
    const int i = li & 15;
    T ar0 = 0, ai0 = 0, ar1 = 0, ai1 = 0;
    // The first group stages the near-field blocks and inputs in shared memory
    // (and loads the epilogue's v, q); then every group applies one row of
    // near offsets.  Only then does the kernel wait for the launch before it
    // (the fused far field, whose CTAs let this grid start as they retire) and
    // apply the far field: the composed L2L and L2P (second group), L2P (third).
    double2 vv = make_double2(0, 0);
    double qq = 0;
    // bulk copies: thread 0 the near blocks, thread 1 + l the far-field blocks
    // of leaf l (static operators, staged when fcc or fcl > 0)
    __shared__ __align__(8) unsigned long long s_bar;
    if (threadIdx.x == 0) {
        mbar_init(&s_bar, 1 + kLeafPerCta);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bulk_expect_copy(sn, near, 9 * 256 * (unsigned)sizeof(C), &s_bar);
        mbar_arrive1(&s_bar);
    } else if (threadIdx.x <= kLeafPerCta) {
        const int l = threadIdx.x - 1, lf = q0 + l;
        if (staged) {
            int ne = 0, coff = 0, nl = 0;
            if (lf < nleaf && c_rowptr != nullptr)
                for (int e = c_rowptr[lf]; e < c_rowptr[lf + 1]; e++, ne++) {
                    const int ri = c_rin[e];
                    if (ri > 0) bulk_expect_copy(sUc + (size_t)(l * fcc + coff) * 16, cm + c_moff[e], 16 * ri * (unsigned)sizeof(C), &s_bar);
                    s_ecol[l][ne] = c_col[e];
                    s_erin[l][ne] = ri;
                    s_ecoff[l][ne] = coff;
                    coff += ri;
                }
            if (lf < nleaf && l2p_rowptr != nullptr && l2p_rowptr[lf + 1] > l2p_rowptr[lf]) {
                const int e = l2p_rowptr[lf];
                nl = l2p_rin[e];
                if (nl > 0) bulk_expect_copy(sUl + (size_t)l * fcl * 16, l2p + l2p_moff[e], 16 * nl * (unsigned)sizeof(C), &s_bar);
            }
            s_nce[l] = ne;
            s_ncc[l] = coff;
            s_nl[l] = nl;
        }
        mbar_arrive1(&s_bar);
    }
    if (grp == 0) {
        const int t0 = li;  // 0 .. 16 kLeafPerCta - 1
        constexpr int kThr = 16 * kLeafPerCta;
        if (leaf < nleaf && q != nullptr) {
            vv = v[(size_t)leaf * 16 + i];
            qq = q[(size_t)leaf * 16 + i];
        }
        for (int t = t0; t < 256; t += kThr) {
            // block position (bx, by) seen from quad leaf l = (bx >= 2) + 2 (by >= 2) at offset (sx, sy)
            const int pos = t >> 4, j = t & 15;
            const int bx = pos & 3, by = pos >> 2;
            const int l = (bx >= 2 ? 1 : 0) | (by >= 2 ? 2 : 0);
            const int sx = bx - 1 - (l & 1), sy = by - 1 - (l >> 1);
            const int src = q0 + l < nleaf ? nbr[(q0 + l) * 9 + (sy + 1) * 3 + (sx + 1)] : -1;
            C val;
            val.x = 0;
            val.y = 0;
            if (src >= 0) {
                if constexpr (sizeof(T) == 8)
                    val = df_split(v[(size_t)src * 16 + j]);  // float pairs, see below
                else
                    val = rnd(v[(size_t)src * 16 + j]);
            }
            vq[pos][j] = val;
        }
    } else if (!staged && leaf < nleaf) {
        // meanwhile the far-field groups bring their operator blocks (static)
        // into L2, so that after the wait only the locals come from afar
        const bool composed = grp == 1;
        const int* rowptr = composed ? c_rowptr : l2p_rowptr;
        if (rowptr != nullptr)
            for (int e = rowptr[leaf]; e < rowptr[leaf + 1]; e++) {
                const C* U = composed ? cm + c_moff[e] : l2p + l2p_moff[e];
                const int ri = composed ? c_rin[e] : l2p_rin[e];
                for (int off = i * 128; off < 16 * ri * (int)sizeof(C); off += 16 * 128)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"((const char*)U + off));
            }
    }
    // the copies have landed (a wait that gives up flags the error and waits once more)
    if (!mbar_wait(&s_bar, 0)) {
        atomicExch(err, 1);
        mbar_wait(&s_bar, 0);
    }
    __syncthreads();
    if (leaf < nleaf) {
        const int l = leaf - q0;
        // complex128: the near blocks and inputs are float pairs, multiplied in double-float
        float dh[2] = {0.f, 0.f}, dl[2] = {0.f, 0.f}, eh[2] = {0.f, 0.f}, el[2] = {0.f, 0.f};
#pragma unroll
        for (int sx = 0; sx < 3; sx++) {
            const int o = grp * 3 + sx;  // offset (sx - 1, grp - 1); outside the domain vq holds zeros
            const C* vs = vq[(1 + (l >> 1) + grp - 1) * 4 + 1 + (l & 1) + sx - 1];
            const C* B = sn + o * 256 + i;
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                if constexpr (sizeof(T) == 8) {
                    df_cmac(dh[0], dl[0], eh[0], el[0], as_df(B[j * 16]), as_df(vs[j]));
                    df_cmac(dh[1], dl[1], eh[1], el[1], as_df(B[(j + 1) * 16]), as_df(vs[j + 1]));
                } else {
                    cmac<T>(ar0, ai0, B[j * 16], vs[j]);
                    cmac<T>(ar1, ai1, B[(j + 1) * 16], vs[j + 1]);
                }
            }
        }
        if constexpr (sizeof(T) == 8) {
            ar1 += ((double)dh[0] + (double)dl[0]) + ((double)dh[1] + (double)dl[1]);
            ai1 += ((double)eh[0] + (double)el[0]) + ((double)eh[1] + (double)el[1]);
        }
    }
    // the far field reads what the launch before wrote (a no-op without a programmatic dependency)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (done != nullptr && blockIdx.x == 0 && threadIdx.x <= kMaxPass) done[threadIdx.x * kDoneStride] = 0;
    if (staged) {
        // the locals of the staged columns (every load in flight at once), then
        // the products from shared memory
        constexpr int kPer = kLeafStageCols / 16;
        const int l = leaf - q0;
        if (grp != 0 && leaf < nleaf) {
            const bool composed = grp == 1;
            const int nc = composed ? s_ncc[l] : s_nl[l];
            C w[kPer], w2[kPer];
            bool two[kPer];
#pragma unroll
            for (int m = 0; m < kPer; m++) {
                const int c = i + 16 * m;
                two[m] = false;
                if (c < nc) {
                    const C *a = nullptr, *a2 = nullptr;
                    if (composed) {
                        int k = 0;
                        while (k + 1 < s_nce[l] && s_ecoff[l][k + 1] <= c) k++;
                        const size_t o = (size_t)s_ecol[l][k] * ldc + (c - s_ecoff[l][k]);
                        a = lcA + o;
                        a2 = lcB ? lcB + o : nullptr;
                    } else {
                        a = lc + (size_t)leaf * ldl + c;
                        a2 = lc2 ? lc2 + (size_t)leaf * ldl + c : nullptr;
                    }
                    w[m] = *a;
                    if (a2) {
                        w2[m] = *a2;
                        two[m] = true;
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < kPer; m++) {
                const int c = i + 16 * m;
                if (c < nc) {
                    C x = w[m];
                    if (two[m]) {
                        if constexpr (sizeof(T) == 8) {
                            x = df_bits(df4_add(as_df(x), as_df(w2[m])));
                        } else {
                            x.x += w2[m].x;
                            x.y += w2[m].y;
                        }
                    }
                    (composed ? suc + l * fcc : sul + l * fcl)[c] = x;
                }
            }
        }
        __syncthreads();
        if (grp != 0 && leaf < nleaf) {
            const bool composed = grp == 1;
            const int nc = composed ? s_ncc[l] : s_nl[l];
            const C* U = composed ? sUc + (size_t)l * fcc * 16 + i : sUl + (size_t)l * fcl * 16 + i;
            const C* u = composed ? suc + l * fcc : sul + l * fcl;
            float dh[2] = {0.f, 0.f}, dl[2] = {0.f, 0.f}, eh[2] = {0.f, 0.f}, el[2] = {0.f, 0.f};
            int c = 0;
            for (; c + 1 < nc; c += 2) {
                if constexpr (sizeof(T) == 8) {
                    df_cmac(dh[0], dl[0], eh[0], el[0], as_df(U[c * 16]), as_df(u[c]));
                    df_cmac(dh[1], dl[1], eh[1], el[1], as_df(U[(c + 1) * 16]), as_df(u[c + 1]));
                } else {
                    cmac<T>(ar0, ai0, U[c * 16], u[c]);
                    cmac<T>(ar1, ai1, U[(c + 1) * 16], u[c + 1]);
                }
            }
            if (c < nc) {
                if constexpr (sizeof(T) == 8)
                    df_cmac(dh[0], dl[0], eh[0], el[0], as_df(U[c * 16]), as_df(u[c]));
                else
                    cmac<T>(ar0, ai0, U[c * 16], u[c]);
            }
            if constexpr (sizeof(T) == 8) {
                ar0 += ((double)dh[0] + (double)dl[0]) + ((double)dh[1] + (double)dl[1]);
                ai0 += ((double)eh[0] + (double)el[0]) + ((double)eh[1] + (double)el[1]);
            }
        }
    } else if (grp != 0 && leaf < nleaf) {
        const bool composed = grp == 1;
        const int* rowptr = composed ? c_rowptr : l2p_rowptr;
        if (rowptr != nullptr) {
            // complex128: operators and locals are float pairs, multiplied in double-float
            // (two column streams), rounded to double once at the end
            float dh[2] = {0.f, 0.f}, dl[2] = {0.f, 0.f}, eh[2] = {0.f, 0.f}, el[2] = {0.f, 0.f};
            for (int e = rowptr[leaf]; e < rowptr[leaf + 1]; e++) {
                // composed: 16 x ri blocks on the parent level's locals (lcA + lcB); L2P: on the leaf's locals
                const C* U = composed ? cm + c_moff[e] + i : l2p + l2p_moff[e] + i;
                const C* u = composed ? lcA + (size_t)c_col[e] * ldc : lc + (size_t)leaf * ldl;
                const C* u2 = composed ? (lcB ? lcB + (size_t)c_col[e] * ldc : nullptr) : (lc2 ? lc2 + (size_t)leaf * ldl : nullptr);
                const int ri = composed ? c_rin[e] : l2p_rin[e];
                // 16 columns at a time, unrolled so that every load issues before the first use
                for (int j0 = 0; j0 < ri; j0 += 16) {
                    C uj[16], Uj[16];
#pragma unroll
                    for (int j = 0; j < 16; j++)
                        if (j0 + j < ri) {
                            uj[j] = u[j0 + j];
                            Uj[j] = U[(j0 + j) * 16];
                            if (u2) {
                                const C w = u2[j0 + j];
                                if constexpr (sizeof(T) == 8) {
                                    uj[j] = df_bits(df4_add(as_df(uj[j]), as_df(w)));
                                } else {
                                    uj[j].x += w.x;
                                    uj[j].y += w.y;
                                }
                            }
                        }
#pragma unroll
                    for (int j = 0; j < 16; j++)
                        if (j0 + j < ri) {
                            if constexpr (sizeof(T) == 8)
                                df_cmac(dh[j & 1], dl[j & 1], eh[j & 1], el[j & 1], as_df(Uj[j]), as_df(uj[j]));
                            else if (j & 1)
                                cmac<T>(ar1, ai1, Uj[j], uj[j]);
                            else
                                cmac<T>(ar0, ai0, Uj[j], uj[j]);
                        }
                }
            }
            if constexpr (sizeof(T) == 8) {
                ar0 += ((double)dh[0] + (double)dl[0]) + ((double)dh[1] + (double)dl[1]);
                ai0 += ((double)eh[0] + (double)el[0]) + ((double)eh[1] + (double)el[1]);
            }
        }
    }
    C mine;
    mine.x = ar0 + ar1;
    mine.y = ai0 + ai1;
    if (grp > 0) part[grp - 1][li] = mine;
    __syncthreads();
    if (grp == 0 && leaf < nleaf) {
        const C a = part[0][li], b = part[1][li];
        const T sr = mine.x + a.x + b.x, si = mine.y + a.y + b.y;
        const size_t gi = (size_t)leaf * 16 + i;
        const double sc = q != nullptr ? k2 * qq : 1.0;  // q == nullptr: the potential K v alone
        out[gi] = make_double2(vv.x + sc * (double)sr, vv.y + sc * (double)si);
    }
}

__global__ void to_c64_kernel(long n, const double2* __restrict__ a, float2* __restrict__ b)
{
    long k = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (k < n) b[k] = make_float2((float)a[k].x, (float)a[k].y);
}

// complex128 as float pairs {re hi, im hi, re lo, im lo}
__global__ void to_df_kernel(long n, const double2* __restrict__ a, double2* __restrict__ b)
{
    long k = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (k < n) b[k] = df_split(a[k]);
}

#define CK(x)                                                                                     \
    do {                                                                                          \
        cudaError_t e_ = (x);                                                                     \
        if (e_ != cudaSuccess) {                                                                  \
            cudaGetLastError(); /* do not leave the error for a later check */                    \
            fail(DAFMM_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_));                   \
        }                                                                                         \
    } while (0)

template <typename P>
void dev_alloc(P** p, size_t bytes)
{
    if (bytes == 0) {
        *p = nullptr;
        return;
    }
    if (cudaMalloc((void**)p, bytes) != cudaSuccess) {
        cudaGetLastError();
        fail(DAFMM_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
}

template <typename V>
void upload_vec(const std::vector<V>& h, V** d)
{
    dev_alloc(d, sizeof(V) * h.size());
    if (!h.empty()) CK(cudaMemcpy(*d, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice));
}

void upload_bsr(BsrHost& h, BsrDev& d)
{
    d.nrows = h.nrows;
    d.Rout = h.Rout;
    d.Rin = h.Rin;
    d.nnz = h.nnz();
    d.nelem = (long)h.mats.size();
    upload_vec(h.rowptr, &d.rowptr);
    upload_vec(h.rout, &d.rout);
    upload_vec(h.col, &d.col);
    upload_vec(h.rin, &d.rin);
    upload_vec(h.moff, &d.moff);
    const size_t n = h.mats.size();
    // two spare entries: a bulk copy rounds its window out to 16-byte words
    dev_alloc((float2**)&d.m32, sizeof(float2) * (n + 4));
    dev_alloc((float4**)&d.mdf, sizeof(float4) * (n + 2));
    CK(cudaMemset(d.m32, 0, sizeof(float2) * (n + 4)));
    CK(cudaMemset(d.mdf, 0, sizeof(float4) * (n + 2)));
    if (n) {
        std::vector<float2> f(n);
        for (size_t k = 0; k < n; k++) f[k] = make_float2((float)h.mats[k].real(), (float)h.mats[k].imag());
        CK(cudaMemcpy(d.m32, f.data(), sizeof(float2) * n, cudaMemcpyHostToDevice));
        std::vector<float2>().swap(f);
        // each double as hi + lo: hi its nearest float, lo the nearest float of the rest
        std::vector<float4> df(n);
        for (size_t k = 0; k < n; k++) {
            const double re = h.mats[k].real(), im = h.mats[k].imag();
            const float rh = (float)re, ih = (float)im;
            df[k] = make_float4(rh, ih, (float)(re - (double)rh), (float)(im - (double)ih));
        }
        CK(cudaMemcpy(d.mdf, df.data(), sizeof(float4) * n, cudaMemcpyHostToDevice));
    }
    std::vector<cd>().swap(h.mats);
}

void free_bsr(BsrDev& d)
{
    cudaFree(d.rowptr);
    cudaFree(d.rout);
    cudaFree(d.col);
    cudaFree(d.rin);
    cudaFree(d.moff);
    cudaFree(d.m32);
    cudaFree(d.mdf);
    d = BsrDev();
}

// Chunk records of one pass, row by row, and the pass's tables.  Every
// row's matrix (rout x J, the row's blocks side by side) is cut into column
// ranges of at most kChunkElems entries and kMaxChunkCols columns.  Record
// b.z / b.w (the row's chunk range in the final list) are filled in when the
// rows are placed.  ldx: stride of the pass's input buffer.
struct PassCut {
    std::vector<int4> recs;     // two int4 per chunk, rows in order
    std::vector<int> first;     // per row: its first record pair in recs (nrows + 1 entries)
    std::vector<long> rbase;
    std::vector<int> cbase, xmap;
    int pld = 0;
};

PassCut cut_pass(const BsrHost& b, int pass, int ldx, int accumulate, const std::vector<char>* initialized, int max_cols = kMaxChunkCols,
                 long max_elems = kChunkElems)
{
    PassCut pc;
    pc.rbase.assign(b.nrows, 0);
    pc.cbase.assign(b.nrows + 1, 0);
    pc.first.assign(b.nrows + 1, 0);
    for (int r = 0; r < b.nrows; r++) {
        pc.first[r] = (int)(pc.recs.size() / 2);
        const int ro = b.rout[r];
        if (b.rowptr[r + 1] > b.rowptr[r]) pc.rbase[r] = b.moff[b.rowptr[r]];
        for (int e = b.rowptr[r]; e < b.rowptr[r + 1]; e++)
            for (int k = 0; k < b.rin[e]; k++) pc.xmap.push_back(b.col[e] * ldx + k);
        pc.cbase[r + 1] = (int)pc.xmap.size();
        if (ro <= 0) continue;
        if (ro > 128) fail(DAFMM_EBADARG, "rank above 128; set max_rank or loosen eps_nca");
        pc.pld = std::max(pc.pld, ro);
        const int J = pc.cbase[r + 1] - pc.cbase[r];
        const int ldr = b.ld[r];
        const int per = (int)std::max<long>(1, std::min<long>(max_cols, max_elems / ldr));
        const int nck = (J + per - 1) / per;
        // add to y only where this application already wrote the row
        const int add = (accumulate && (!initialized || (*initialized)[r])) ? kFlagAddHost : 0;
        for (int j = 0; j < J; j += per) {
            const int j1 = std::min(J, j + per);
            const long elem = pc.rbase[r] + (long)j * ldr;
            pc.recs.push_back(make_int4(pass | add | (nck == 1 ? kFlagDirectHost : 0) | (ro << 16), r, j1 - j, pc.cbase[r] + j));
            pc.recs.push_back(make_int4((int)(elem & 0xffffffffL), (int)(elem >> 32), 0, 0));
        }
    }
    pc.first[b.nrows] = (int)(pc.recs.size() / 2);
    return pc;
}

// Append row r of a cut pass to the list, with its chunk range.
// A chunk whose matrix equals an earlier chunk's of the same pass, entry for
// entry as stored (complex64 when `c64`, else complex128), takes the earlier
// chunk's address: the same products from the same numbers.  On a uniform
// grid the entry table depends only on the offset between boxes, so boxes
// with the same neighbourhood get the same blocks; the copies then come
// from L2 instead of DRAM.
void dedup_chunks(std::vector<int4>& recs, const std::vector<const BsrHost*>& hs, bool c64)
{
    std::vector<std::unordered_map<unsigned long long, std::vector<long>>> seen(hs.size());
    auto entry = [&](const BsrHost& B, long elem, long k, unsigned (&w)[4]) {
        const cd z = B.mats[elem + k];
        if (c64) {
            const float re = (float)z.real(), im = (float)z.imag();
            std::memcpy(&w[0], &re, 4);
            std::memcpy(&w[1], &im, 4);
            w[2] = w[3] = 0;
        } else {
            const double re = z.real(), im = z.imag();
            std::memcpy(&w[0], &re, 8);
            std::memcpy(&w[2], &im, 8);
        }
    };
    const long nch = (long)(recs.size() / 2);
    for (long c = 0; c < nch; c++) {
        const int4 a = recs[2 * c];
        int4& b = recs[2 * c + 1];
        const int p = a.x & 0xff;
        const BsrHost& B = *hs[p];
        const int ro = (a.x >> 16) & 0xffff;
        const long n = (long)(ro + (ro & 1)) * a.z;
        const long elem = (long)(unsigned)b.x | ((long)b.y << 32);
        unsigned long long h = 1469598103934665603ull ^ ((unsigned long long)ro << 32 | (unsigned)a.z);
        for (long k = 0; k < n; k++) {
            unsigned w[4];
            entry(B, elem, k, w);
            for (unsigned x : w) h = (h ^ x) * 1099511628211ull;
        }
        long same = -1;
        for (long e : seen[p][h]) {
            bool eq = true;
            for (long k = 0; k < n && eq; k++) {
                unsigned w1[4], w2[4];
                entry(B, elem, k, w1);
                entry(B, e, k, w2);
                eq = std::memcmp(w1, w2, sizeof(w1)) == 0;
            }
            if (eq) {
                same = e;
                break;
            }
        }
        if (same < 0) {
            seen[p][h].push_back(elem);
        } else {
            b.x = (int)(unsigned)(same & 0xffffffffL);
            b.y = (int)(same >> 32);
        }
    }
}

void place_row(std::vector<int4>& out, const PassCut& pc, int r)
{
    const int c0 = (int)(out.size() / 2);
    const int n = pc.first[r + 1] - pc.first[r];
    for (int k = 0; k < n; k++) {
        out.push_back(pc.recs[2 * (pc.first[r] + k)]);
        int4 b = pc.recs[2 * (pc.first[r] + k) + 1];
        b.z = c0 + n;
        b.w = c0;
        out.push_back(b);
    }
}

void upload_tables(Group& g, const PassCut& pc)
{
    long* drb = nullptr;
    int* dcb = nullptr;
    int* dxm = nullptr;
    upload_vec(pc.rbase, &drb);
    upload_vec(pc.cbase, &dcb);
    upload_vec(pc.xmap, &dxm);
    g.rbase.push_back(drb);
    g.cbase.push_back(dcb);
    g.xmap.push_back(dxm);
    g.xmap_n.push_back((int)pc.xmap.size());
}

void finish_group(Group& g, const std::vector<int4>& recs, int pld)
{
    g.nch = (int)(recs.size() / 2);
    g.Pld = std::max(pld, 1);
    upload_vec(recs, &g.chunks);
    std::vector<int> zeros(std::max(g.nch, 1), 0);
    upload_vec(zeros, &g.cnt);
}

// Passes launched together (several right-hand sides): rows in order.
void build_group(Group& g, const std::vector<PassRef>& passes, const std::vector<const BsrHost*>& hs, const std::vector<int>& ldx,
                 int accumulate, const std::vector<char>* initialized = nullptr)
{
    if (passes.size() > (size_t)kMaxPass) fail(DAFMM_EBADARG, "too many passes in one launch group");
    g.passes = passes;
    g.accumulate = accumulate;
    std::vector<int4> recs;
    int pld = 0;
    for (size_t p = 0; p < hs.size(); p++) {
        const PassCut pc = cut_pass(*hs[p], (int)p, ldx[p], accumulate, initialized, kMaxChunkColsB);
        for (int r = 0; r < hs[p]->nrows; r++) place_row(recs, pc, r);
        pld = std::max(pld, pc.pld);
        upload_tables(g, pc);
    }
    finish_group(g, recs, pld);
}

// Persistent CTAs of the fused kernel on this device.
template <typename T>
int fused_ctas()
{
    int dev = 0, sms = 0, per_sm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_kernel<T>, 32 * kStreamWarps, StreamCfg<T>::kCta));
    return std::max(1, sms * std::max(per_sm, 1));
}

// C = A B for column-major blocks: A is m x k (column stride lda), B is k x n
// (column stride ldb), C is m x n (column stride ldc).
void block_mul(const cd* A, int lda, const cd* B, int ldb, cd* C, int ldc, int m, int k, int n)
{
    for (int j = 0; j < n; j++)
        for (int i = 0; i < m; i++) {
            cd s = 0;
            for (int l = 0; l < k; l++) s += A[(size_t)l * lda + i] * B[(size_t)j * ldb + l];
            C[(size_t)j * ldc + i] = s;
        }
}

// The up pass of level L-1 composed with the leaves' P2M: every block
// T_e (ro x ro_c, child leaf c) becomes T_e V_c (ro x 16), V_c the P2M block
// of leaf c, so the multipoles of level L-1 come straight from the leaf values.
BsrHost compose_up(const BsrHost& T, const BsrHost& V)
{
    BsrHost C;
    C.nrows = T.nrows;
    C.Rout = T.Rout;
    C.Rin = 16;
    C.rowptr = T.rowptr;
    C.rout = T.rout;
    C.col.resize(T.col.size());
    C.rin.assign(T.col.size(), 16);
    for (size_t e = 0; e < T.col.size(); e++) {
        const int c = T.col[e];
        C.col[e] = c;  // leaf slot = leaf
        if (T.rin[e] == 0) continue;
        if (V.rowptr[c + 1] - V.rowptr[c] != 1 || V.rin[V.rowptr[c]] != 16 || V.rout[c] != T.rin[e] || V.col[V.rowptr[c]] != c)
            fail(DAFMM_EBADARG, "composing P2M: a leaf row is not one 16-column block of the child's rank");
    }
    C.layout();
    for (int r = 0; r < T.nrows; r++)
        for (int e = T.rowptr[r]; e < T.rowptr[r + 1]; e++) {
            const int c = T.col[e];
            if (T.rin[e] == 0 || T.rout[r] == 0) continue;  // zero block (layout zeroes mats)
            const int ev = V.rowptr[c];
            block_mul(&T.mats[T.moff[e]], T.ld[r], &V.mats[V.moff[ev]], V.ld[c], &C.mats[C.moff[e]], C.ld[r], T.rout[r], T.rin[e], 16);
        }
    return C;
}

// The L2L into the leaves composed with their L2P: every block D_e (ri_b x
// ri_s, parent slot s) of leaf b becomes U_b D_e (16 x ri_s), U_b the L2P
// block of leaf b, so the leaf values come straight from the parent's locals.
BsrHost compose_leaf(const BsrHost& D, const BsrHost& U)
{
    BsrHost C;
    C.nrows = D.nrows;
    C.Rout = 16;
    C.Rin = D.Rin;
    C.rowptr = D.rowptr;
    C.col = D.col;
    C.rin = D.rin;
    C.rout.assign(D.nrows, 0);
    for (int b = 0; b < D.nrows; b++) {
        if (D.rowptr[b + 1] == D.rowptr[b]) continue;
        C.rout[b] = 16;
        if (D.rout[b] == 0) continue;
        if (U.rowptr[b + 1] - U.rowptr[b] != 1 || U.rout[b] != 16 || U.rin[U.rowptr[b]] != D.rout[b])
            fail(DAFMM_EBADARG, "composing L2P: a leaf row is not one 16-row block of the leaf's rank");
    }
    C.layout();
    for (int b = 0; b < D.nrows; b++) {
        if (D.rout[b] == 0) continue;  // zero blocks (layout zeroes mats)
        for (int e = D.rowptr[b]; e < D.rowptr[b + 1]; e++) {
            const int eu = U.rowptr[b];
            block_mul(&U.mats[U.moff[eu]], U.ld[b], &D.mats[D.moff[e]], D.ld[b], &C.mats[C.moff[e]], C.ld[b], 16, D.rout[b], D.rin[e]);
        }
    }
    return C;
}

// Warp shares of a plan's chain list for a grid of `warps` warps (each phase
// shared by F.wn[k] of them when the plan sets them): chunks per warp in each
// phase, and the shares in the phases before.  Returns the shares.
int fused_shares(const FusedPlan& F, int warps, int* kpw, int* sbase)
{
    int n = 0;
    for (int k = 0; k < F.nph; k++) {
        const int nk = F.base[k + 1] - F.base[k];
        const int nw = F.wn.empty() ? warps : std::max(1, F.wn[k]);
        kpw[k] = std::max(1, (nk + nw - 1) / nw);
        sbase[k] = n;
        n += (nk + kpw[k] - 1) / kpw[k];
    }
    return n;
}

// The fused single-right-hand-side launch.  Passes, in an order where every
// pass comes after those it reads: up at levels L..top, M2L at top..L, down
// at top..L-1 (the down pass of level nu reads the M2L locals and the
// parent's down output of level nu and writes its own buffer for level nu+1).
// A pass's earliest phase (asap) is one more than the latest of the passes it
// reads, its latest (alap) one less than the earliest of its readers; passes
// with alap > asap (M2L below the top level) have slack, and every pass they
// read is on the chain.  Every row a chunk reads lies in an earlier phase (or
// in a bulk pass whose inputs do), and a warp works through its shares phase
// by phase, so the waits cannot form a cycle.
void build_fused(const Tree& t, const OpsHost& h, OpsDev& d, const BsrHost* upc)
{
    Fused& F = d.fz;
    const int L = t.L, top = t.top;
    std::vector<PassRef> passes;
    std::vector<const BsrHost*> hs;
    std::vector<int> ldx;
    std::vector<unsigned> deps;
    std::vector<int> up_i(L + 1, -1), m2l_i(L + 1, -1), down_i(L + 1, -1);
    for (int nu = L; nu >= top; nu--) {
        up_i[nu] = (int)passes.size();
        if (nu == L - 1 && upc) {
            // multipoles of level L-1 straight from the leaf values
            passes.push_back(PassRef{nu, 3});
            hs.push_back(upc);
            ldx.push_back(16);
            deps.push_back(0u);
            continue;
        }
        passes.push_back(PassRef{nu, 0});
        hs.push_back(&h.lv[nu].up);
        ldx.push_back(nu == L ? 16 : h.lv[nu + 1].Ro);
        deps.push_back(nu == L ? 0u : 1u << up_i[nu + 1]);
    }
    for (int nu = top; nu <= L; nu++) {
        m2l_i[nu] = (int)passes.size();
        passes.push_back(PassRef{nu, 1});
        hs.push_back(&h.lv[nu].m2l);
        ldx.push_back(h.lv[nu].Ro);
        deps.push_back(1u << up_i[nu]);
    }
    // the L2L from level L-1 is composed with L2P in the leaf kernel
    for (int nu = top; nu < L - 1; nu++) {
        down_i[nu] = (int)passes.size();
        passes.push_back(PassRef{nu, 2});
        hs.push_back(&h.lv[nu].down);
        ldx.push_back(h.lv[nu].Ri);
        deps.push_back((1u << m2l_i[nu]) | (nu > top ? 1u << down_i[nu - 1] : 0u));
    }
    const int np = (int)passes.size();
    if (np > kMaxPass) fail(DAFMM_EBADARG, "too many far-field levels for the fused launch");
    // chunk records of plan 0 (complex128) and plan 1 (complex64); the row and
    // column tables do not depend on the chunk size
    std::vector<PassCut> cuts_k[2];
    int pld = 0;
    for (int p = 0; p < np; p++) {
        cuts_k[0].push_back(cut_pass(*hs[p], p, ldx[p], 0, nullptr, kMaxChunkCols, StreamCfg<double>::kElems));
        cuts_k[1].push_back(cut_pass(*hs[p], p, ldx[p], 0, nullptr, kMaxChunkCols, StreamCfg<float>::kElems));
        pld = std::max(pld, cuts_k[1][p].pld);
    }
    const std::vector<PassCut>& cuts = cuts_k[1];
    std::vector<int> asap(np, 0), alap(np, 0);
    for (int p = 0; p < np; p++)
        for (int q = 0; q < p; q++)
            if (deps[p] >> q & 1u) asap[p] = std::max(asap[p], asap[q] + 1);
    int nph = 0;
    for (int p = 0; p < np; p++) nph = std::max(nph, asap[p] + 1);
    if (nph > kMaxPhase) fail(DAFMM_EBADARG, "too many phases for the fused launch");
    for (int p = 0; p < np; p++) {
        alap[p] = nph - 1;
        for (int r = p + 1; r < np; r++)
            if (deps[r] >> p & 1u) alap[p] = std::min(alap[p], asap[r] - 1);
    }
    auto chunks_in = [&](int k, int p, int r) { return cuts_k[k][p].first[r + 1] - cuts_k[k][p].first[r]; };
    auto chunks = [&](int p, int r) { return chunks_in(1, p, r); };
    std::vector<char> slack(np, 0);
    for (int p = 0; p < np; p++) slack[p] = alap[p] > asap[p];
    F.dphase.assign(np, -1);
    for (int p = 0; p < np; p++)
        for (int q = 0; q < np; q++)
            if (deps[p] >> q & 1u) {
                if (slack[p] && slack[q]) fail(DAFMM_EBADARG, "fused launch: a pass with slack reads another");
                F.dphase[p] = std::max(F.dphase[p], asap[q]);
            }
    F.g.Pld = std::max(pld, 1);
    for (int k = 0; k < 2; k++) {
        FusedPlan& P = F.plan[k];
        const bool dynamic = k == 0 ? kPieces128 : kPieces64;
        const bool split = k == 0 ? kSplit128 : kSplit64;
        auto chunks = [&](int p, int r) { return chunks_in(k, p, r); };
        const std::vector<PassCut>& cuts = cuts_k[k];
        // rows of every chain phase, each pass at its earliest phase
        std::vector<std::vector<std::pair<int, int>>> rows(nph);
        for (int p = 0; p < np; p++)
            if (!slack[p])
                for (int r = 0; r < hs[p]->nrows; r++)
                    if (chunks(p, r)) rows[asap[p]].push_back({p, r});
        // the static plan: after each chain phase, one phase per slack pass
        // whose inputs it completes (finest level first).  The first phase is
        // shared by every warp; then the chain phases by the first wc warps
        // and the slack phases by the others, so that the slack passes stream
        // while the chain steps through its dependent passes
        std::vector<char> bulk_ph(nph, 0);
        if (!dynamic) {
            std::vector<std::vector<std::pair<int, int>>> out;
            std::vector<char> is_bulk;
            for (int ph = 0; ph < nph; ph++) {
                out.push_back(rows[ph]);
                is_bulk.push_back(0);
                std::vector<int> sl;
                for (int p = 0; p < np; p++)
                    if (slack[p] && std::max(F.dphase[p], 0) == ph) sl.push_back(p);
                std::stable_sort(sl.begin(), sl.end(), [&](int a, int b) { return passes[a].level > passes[b].level; });
                for (int p : sl) {
                    out.emplace_back();
                    for (int r = 0; r < hs[p]->nrows; r++)
                        if (chunks(p, r)) out.back().push_back({p, r});
                    is_bulk.push_back(1);
                }
            }
            rows.swap(out);
            bulk_ph.swap(is_bulk);
        }
        const int nphase = (int)rows.size();
        if (nphase > kMaxPhase) fail(DAFMM_EBADARG, "too many phases for the fused launch");
        std::vector<int4> recs;
        P.nph = nphase;
        P.base.assign(nphase + 1, 0);
        P.phdeps.assign(nphase, 0u);
        long after0[2] = {0, 0};  // chunks after the first phase: chain, slack
        for (int ph = 0; ph < nphase; ph++) {
            P.base[ph] = (int)(recs.size() / 2);
            for (auto& pr : rows[ph]) {
                P.phdeps[ph] |= deps[pr.first];
                place_row(recs, cuts[pr.first], pr.second);
            }
            if (ph > 0) after0[bulk_ph[ph]] += (long)(recs.size() / 2) - P.base[ph];
        }
        P.base[nphase] = (int)(recs.size() / 2);
        if (dynamic)
            for (int p = 0; p < np; p++)
                if (slack[p])
                    for (int r = 0; r < hs[p]->nrows; r++) after0[1] += chunks(p, r);
        P.wlo.clear();
        P.wn.clear();
        P.chain_split = split && dynamic;
        if (split) {
            const int W = F.ctas[k] * kStreamWarps;
            int wc = W;  // chain warps
            if (after0[1] == 0)
                wc = W;
            else if (after0[0] == 0)
                wc = 0;
            else
                wc = std::min(W - 1, std::max(1, (int)std::lround(W * (k == 0 ? kChainShare128 : kChainShare64) * after0[0] /
                                                                  (double)(after0[0] + after0[1]))));
            for (int ph = 0; ph < nphase; ph++) {
                const bool all = ph == 0 || (bulk_ph[ph] ? wc == 0 : wc == W);
                P.wlo.push_back(all ? 0 : (bulk_ph[ph] ? wc : 0));
                P.wn.push_back(all ? W : (bulk_ph[ph] ? W - wc : wc));
            }
        }
        int kpw[kMaxPhase], sbase[kMaxPhase];
        const int chain_slots = fused_shares(P, F.ctas[k] * kStreamWarps, kpw, sbase);
        // dynamic plan: the slack passes as pieces of kPiece chunks, earliest inputs first
        std::vector<int4> pieces;
        if (dynamic) {
            std::vector<int> order;
            for (int p = 0; p < np; p++)
                if (slack[p]) order.push_back(p);
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
                const int da = std::max(F.dphase[a], 0), db = std::max(F.dphase[b], 0);
                return da != db ? da < db : passes[a].level > passes[b].level;
            });
            for (int p : order)
                for (int r = 0; r < hs[p]->nrows; r++) {
                    const int n = chunks(p, r);
                    if (!n) continue;
                    const int c0 = (int)(recs.size() / 2);
                    place_row(recs, cuts[p], r);
                    for (int j = 0; j < n; j += kPiece)
                        pieces.push_back(make_int4(c0 + j, c0 + std::min(n, j + kPiece), chain_slots + (int)pieces.size(), p));
                }
        }
        P.npieces = (int)pieces.size();
        if (!pieces.empty()) upload_vec(pieces, &P.pieces);
        P.nch = (int)(recs.size() / 2);
        if (kDedupChunks) dedup_chunks(recs, hs, k == 1);
        upload_vec(recs, &P.chunks);
        std::vector<int> zeros(std::max(P.nch, 1), 0);
        upload_vec(zeros, &P.cnt);
        P.part = (size_t)(chain_slots + P.npieces) * F.g.Pld;
    }
    F.deps = deps;
    F.target.assign(np, 0);
    F.cmacs = 0;
    for (int p = 0; p < np; p++)
        for (int r = 0; r < hs[p]->nrows; r++) {
            F.target[p] += chunks(p, r) > 0;
            F.cmacs += (double)hs[p]->rout[r] * (cuts[p].cbase[r + 1] - cuts[p].cbase[r]);
        }
    F.g.passes = passes;
    F.g.accumulate = 0;
    for (int p = 0; p < np; p++) upload_tables(F.g, cuts[p]);
    std::vector<int> zeros((kMaxPass + 1) * kDoneStride, 0);
    upload_vec(zeros, &F.done);
}

void free_fused(Fused& F)
{
    for (FusedPlan& P : F.plan) {
        cudaFree(P.pieces);
        cudaFree(P.chunks);
        cudaFree(P.cnt);
    }
    for (long* p : F.g.rbase) cudaFree(p);
    for (int* p : F.g.cbase) cudaFree(p);
    for (int* p : F.g.xmap) cudaFree(p);
    cudaFree(F.done);
    F = Fused();
}

void free_group(Group& g)
{
    cudaFree(g.chunks);
    cudaFree(g.cnt);
    for (long* p : g.rbase) cudaFree(p);
    for (int* p : g.cbase) cudaFree(p);
    for (int* p : g.xmap) cudaFree(p);
    g = Group();
}

// Coefficient buffers and chunk partials of one application.
template <typename T>
struct Bufs {
    using C = typename V2<T>::t;
    C* mp[64] = {};
    C* lc[64] = {};
    C* part = nullptr;
};

template <typename T>
PassArgs<T> pass_args(const Tree& t, const OpsDev& d, const Bufs<T>& b, const typename V2<T>::t* vin, const Group& g, int p)
{
    using C = typename V2<T>::t;
    const PassRef& pr = g.passes[p];
    const int nu = pr.level;
    const LevelDev& l = d.lv[nu];
    const BsrDev& bs = pr.kind == 0 ? l.up : (pr.kind == 1 ? l.m2l : l.down);
    PassArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.rout = bs.rout;
    a.rbase = g.rbase[p];
    a.cbase = g.cbase[p];
    a.xmap = g.xmap[p];
    a.mats = (const C*)(sizeof(T) == 8 ? bs.mdf : bs.m32);  // complex128: float pairs
    if (pr.kind == 0) {
        a.x = nu == t.L ? vin : b.mp[nu + 1];
        a.y = b.mp[nu];
        a.ldy = l.Ro;
    } else if (pr.kind == 1) {
        a.x = b.mp[nu];
        a.y = b.lc[nu];
        a.ldy = l.Ri;
    } else {
        a.x = b.lc[nu];
        a.y = b.lc[nu + 1];
        a.ldy = d.lv[nu + 1].Ri;
    }
    return a;
}

// Coefficients of a fused application: multipoles, locals from M2L and
// locals from the parent per level, and the chunk partials.
template <typename T>
struct FBufs {
    using C = typename V2<T>::t;
    C* mp[64] = {};
    C* lc[64] = {};
    C* lcd[64] = {};
    C* part = nullptr;
};

template <typename T>
PassArgs<T> fused_pass_args(const Tree& t, const OpsDev& d, const FBufs<T>& b, const double* v, int p)
{
    using C = typename V2<T>::t;
    const Group& g = d.fz.g;
    const PassRef& pr = g.passes[p];
    const int nu = pr.level;
    const LevelDev& l = d.lv[nu];
    const BsrDev& bs = pr.kind == 0 ? l.up : (pr.kind == 1 ? l.m2l : (pr.kind == 2 ? l.down : l.upc));
    PassArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.rout = bs.rout;
    a.rbase = g.rbase[p];
    a.cbase = g.cbase[p];
    a.xmap = g.xmap[p];
    // complex128: the float-pair copy (16 bytes an entry, like double2), see chunk_mac
    a.mats = (const C*)(sizeof(T) == 8 ? bs.mdf : bs.m32);
    if (pr.kind == 0 || pr.kind == 3) {
        if (nu == t.L || pr.kind == 3)
            a.xd = (const double2*)v;
        else
            a.x = b.mp[nu + 1];
        a.y = b.mp[nu];
        a.ldy = l.Ro;
    } else if (pr.kind == 1) {
        a.x = b.mp[nu];
        a.y = b.lc[nu];
        a.ldy = l.Ri;
    } else {
        a.x = b.lc[nu];
        a.x2 = nu > t.top ? b.lcd[nu] : nullptr;
        a.y = b.lcd[nu + 1];
        a.ldy = d.lv[nu + 1].Ri;
    }
    return a;
}

// One cooperative launch of every tree pass (see stream_kernel).
template <typename T>
void launch_fused(const Tree& t, const OpsDev& d, const FBufs<T>& b, const double* v, cudaStream_t s)
{
    const Fused& F = d.fz;
    const int k = sizeof(T) == 4 ? 1 : 0;
    const FusedPlan& FP = F.plan[k];
    if (FP.nch == 0) return;
    GroupArgs<T> ga;
    std::memset(&ga, 0, sizeof(ga));
    for (size_t p = 0; p < F.g.passes.size(); p++) ga.p[p] = fused_pass_args<T>(t, d, b, v, (int)p);
    const int ctas = F.ctas[k];
    const int warps = ctas * kStreamWarps;
    Sched sc;
    std::memset(&sc, 0, sizeof(sc));
    sc.nph = FP.nph;
    for (int ph = 0; ph <= FP.nph; ph++) sc.base[ph] = FP.base[ph];
    for (int ph = 0; ph < FP.nph; ph++) {
        sc.wlo[ph] = FP.wlo.empty() ? 0 : FP.wlo[ph];
        sc.wn[ph] = FP.wn.empty() ? warps : FP.wn[ph];
    }
    fused_shares(FP, warps, sc.kpw, sc.sbase);
    for (int ph = 0; ph < FP.nph; ph++) sc.phdeps[ph] = FP.phdeps[ph];
    sc.npieces = FP.npieces;
    sc.chain_split = FP.chain_split ? 1 : 0;
    sc.npf = 0;
    sc.pf_ptr[sc.npf] = (const char*)FP.chunks;
    sc.pf_bytes[sc.npf++] = FP.nch * (int)(2 * sizeof(int4));
    for (size_t p = 0; p < F.g.passes.size() && sc.npf <= kMaxPass; p++) {
        sc.pf_ptr[sc.npf] = (const char*)F.g.xmap[p];
        sc.pf_bytes[sc.npf++] = F.g.xmap_n[p] * (int)sizeof(int);
    }
    sc.pieces = FP.pieces;
    sc.next_piece = F.done + kMaxPass * kDoneStride;
    for (size_t p = 0; p < F.g.passes.size(); p++) {
        sc.deps[p] = F.deps[p];
        sc.target[p] = F.target[p];
        sc.dphase[p] = F.dphase[p];
        for (size_t q = 0; q < F.g.passes.size(); q++)
            if (F.deps[q] >> p & 1u) sc.pub |= 1u << p;
    }
    if (d.stall_pass >= 0) sc.target[d.stall_pass] += 1;  // a row nobody writes: the waits on it give up
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(32 * kStreamWarps);
    cfg.dynamicSmemBytes = StreamCfg<T>::kCta;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, stream_kernel<T>, (const int4*)FP.chunks, ga, sc, b.part, F.g.Pld, FP.cnt, F.done, d.err));
}

// Events recorded while a graph is being captured (its five pass marks).
thread_local cudaEvent_t* tl_capture_events = nullptr;

// Record event k (0..4) of the current profiled call on the handle d.
void mark(OpsDev* d, int k, cudaStream_t s)
{
    if (tl_capture_events) {
        // an external record node (a plain record in capture only orders streams)
        CK(cudaEventRecordWithFlags(tl_capture_events[k], s, cudaEventRecordExternal));
        return;
    }
    if (!d || !d->profile) return;
    if (k == 0) {
        if (d->ev_used + 5 > (size_t)5 * 65536) return;
        while (d->events.size() < d->ev_used + 5) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            d->events.push_back(e);
        }
        d->ev_used += 5;
        d->ev_fused.resize(d->ev_used / 5, 0);
    }
    if (d->ev_used < 5) return;
    CK(cudaEventRecord(d->events[d->ev_used - 5 + k], s));
}

// The profiled call whose events were taken last runs the fused far field.
void mark_fused(OpsDev* d)
{
    if (!tl_capture_events && d && d->profile && d->ev_used >= 5) d->ev_fused[d->ev_used / 5 - 1] = 1;
}

// One right-hand side: the fused far field, then the leaf kernel.  prof:
// handle whose events record the passes (nullptr: none); the far field is
// the first interval.
template <typename T>
void run_fused(const Tree& t, const OpsDev& d, const FBufs<T>& b, const double* v, double* out, cudaStream_t s, OpsDev* prof)
{
    using C = typename V2<T>::t;
    const int L = t.L;
    const int nleaf = t.nb * t.nb;
    const bool far = t.top <= L;
    mark(prof, 0, s);
    mark_fused(prof);
    if (far) launch_fused<T>(t, d, b, v, s);
    mark(prof, 1, s);
    mark(prof, 2, s);
    mark(prof, 3, s);
    const C* nearp = (const C*)(sizeof(T) == 8 ? (const void*)d.neardf : (const void*)d.near32);
    const BsrDev* l2p = far ? &d.lv[L].down : nullptr;
    const bool comp = far && L - 1 >= t.top;
    const C* cm = comp ? (const C*)(sizeof(T) == 8 ? d.leafc.mdf : d.leafc.m32) : nullptr;
    // programmatic serialization: the leaf CTAs start (near field) while the
    // far field's CTAs retire, and wait in the kernel for its writes
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)((nleaf + kLeafPerCta - 1) / kLeafPerCta));
    cfg.blockDim = dim3(48 * kLeafPerCta);
    cfg.dynamicSmemBytes = (size_t)kLeafPerCta * 17 * (d.fz.leaf_fcc + d.fz.leaf_fcl) * sizeof(C);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = far ? 1 : 0;
    CK(cudaLaunchKernelEx(&cfg, leaf_apply_kernel<T>, nleaf, (const int*)d.nbr, nearp, l2p ? (const int*)l2p->rowptr : nullptr,
                          l2p ? (const long*)l2p->moff : nullptr, l2p ? (const int*)l2p->rin : nullptr,
                          l2p ? (const C*)(sizeof(T) == 8 ? l2p->mdf : l2p->m32) : nullptr, far ? d.lv[L].Ri : 0,
                          far ? (const C*)b.lc[L] : nullptr, (const C*)nullptr, comp ? (const int*)d.leafc.rowptr : nullptr,
                          comp ? (const int*)d.leafc.col : nullptr, comp ? (const long*)d.leafc.moff : nullptr,
                          comp ? (const int*)d.leafc.rin : nullptr, cm, comp ? d.lv[L - 1].Ri : 0, comp ? (const C*)b.lc[L - 1] : nullptr,
                          comp && L - 1 > t.top ? (const C*)b.lcd[L - 1] : nullptr, (const double2*)v, (const double*)(d.potential ? nullptr : d.q),
                          (double)(t.prm.kappa * t.prm.kappa), (double2*)out, far ? d.fz.done : (int*)nullptr, d.fz.leaf_fcc,
                          d.fz.leaf_fcl, d.err));
    mark(prof, 4, s);
}

template <typename T, int MR>
void launch_batched_mr(const OpsDev& d, const Group& g, const GroupArgs<T>& ga, typename V2<T>::t* part, int nrhs, cudaStream_t s)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int nrhs_pad = (nrhs + kRhsPerWarp - 1) / kRhsPerWarp * kRhsPerWarp;
    const int threads = 32 * (nrhs_pad / kRhsPerWarp);
    const int smem = BatchCfg<T>::cta_bytes(nrhs_pad);
    CK(cudaFuncSetAttribute(stream_batched_kernel<T, MR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_batched_kernel<T, MR>, threads, smem));
    if (d.batched_cps > 0) per_sm = std::min(per_sm, d.batched_cps);  // tuned grid
    per_sm = std::max(per_sm, 1);
    int kpc = 1;
    if (g.nch > 0) {
        const int ctas = std::max(1, std::min(g.nch, sms * per_sm));
        kpc = (g.nch + ctas - 1) / ctas;
        const int grid = (g.nch + kpc - 1) / kpc;
        // inputs by bulk copies when every column is a 16-byte multiple at a 16-byte aligned address
        int bulk_x = (nrhs * (int)sizeof(typename V2<T>::t)) % 16 == 0;
        for (size_t p = 0; p < g.passes.size(); p++) bulk_x &= ((uintptr_t)ga.p[p].x % 16) == 0;
        stream_batched_kernel<T, MR><<<(unsigned)grid, threads, smem, s>>>(g.nch, kpc, nrhs, nrhs_pad, bulk_x, g.chunks, ga, part,
                                                                         g.Pld, g.cnt, d.err);
    }
}

// Several right-hand sides, complex64, on the tensor cores (one CTA per SM:
// its operand buffers take most of the shared memory).
void launch_batched_tc(const OpsDev& d, const Group& g, const GroupArgs<float>& ga, float2* part, int nrhs, cudaStream_t s)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int nrhs_pad = (nrhs + kRhsPerWarp - 1) / kRhsPerWarp * kRhsPerWarp;
    const int smem = tc_smem_bytes(nrhs_pad);
    CK(cudaFuncSetAttribute(stream_batched_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_batched_tc_kernel, kTcThreads, smem));
    per_sm = std::max(per_sm, 1);
    const int ctas = std::max(1, std::min(g.nch, sms * per_sm));
    const int kpc = (g.nch + ctas - 1) / ctas;
    const int grid = (g.nch + kpc - 1) / kpc;
    int bulk_x = (nrhs * (int)sizeof(float2)) % 16 == 0;
    for (size_t p = 0; p < g.passes.size(); p++) bulk_x &= ((uintptr_t)ga.p[p].x % 16) == 0;
    stream_batched_tc_kernel<<<(unsigned)grid, kTcThreads, smem, s>>>(g.nch, kpc, nrhs, nrhs_pad, bulk_x, g.chunks, ga, part, g.Pld, g.cnt,
                                                                      d.err);
}

// Tensor cores for the complex64 several-right-hand-side passes (see
// dafmm_set_batched_kernel).  Automatic mode keeps the CUDA-core kernel: at
// these chunk shapes (M = 128 stacked rows, N = 2 NR <= 128, K <= 64 per
// chunk) the operand conversion and the serial per-chunk steps cost more than
// the FMAs they replace (64 right-hand sides at N = 16384: 1.33 ms on the
// tensor cores, 0.74 ms on the CUDA cores).
constexpr int kTcMinRhs = 8;
constexpr bool kTcAuto = false;

template <typename T>
void launch_group_batched(const Tree& t, const OpsDev& d, const Bufs<T>& b, const typename V2<T>::t* vin, const Group& g, int nrhs,
                          cudaStream_t s)
{
    if (g.nch == 0) return;
    GroupArgs<T> ga;
    std::memset(&ga, 0, sizeof(ga));
    for (size_t p = 0; p < g.passes.size(); p++) ga.p[p] = pass_args<T>(t, d, b, vin, g, (int)p);
    if constexpr (sizeof(T) == 4) {
        const bool tc = d.batched_kernel == 2 || (d.batched_kernel == 0 && kTcAuto && nrhs >= kTcMinRhs);
        if (tc && g.Pld <= 64) {
            launch_batched_tc(d, g, ga, b.part, nrhs, s);
            return;
        }
    }
    const int h = ((g.Pld + 3) >> 2) << 1;  // rows per lane of the widest row
    if (h <= 8)
        launch_batched_mr<T, 8>(d, g, ga, b.part, nrhs, s);
    else if (h <= 16)
        launch_batched_mr<T, 16>(d, g, ga, b.part, nrhs, s);
    else if (h <= 24)
        launch_batched_mr<T, 24>(d, g, ga, b.part, nrhs, s);
    else if (h <= 32)
        launch_batched_mr<T, 32>(d, g, ga, b.part, nrhs, s);
    else
        fail(DAFMM_EBADARG, "ranks above 64 are not supported with several right-hand sides");
}

template <typename T>
void run_batched(const Tree& t, const OpsDev& d, const Bufs<T>& b, float2* v32, const double* v, double* out, int nrhs, cudaStream_t s,
                 OpsDev* prof)
{
    using C = typename V2<T>::t;
    const int L = t.L;
    const long N = t.N;
    const int nleaf = t.nb * t.nb;
    mark(prof, 0, s);
    const C* vin;
    const long nv = N * nrhs;
    if (sizeof(T) == 4) {
        to_c64_kernel<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(nv, (const double2*)v, v32);
        vin = (const C*)v32;
    } else {
        // complex128: every pass and the leaf kernel compute in double-float (see Acc<double>)
        to_df_kernel<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(nv, (const double2*)v, (double2*)d.vdf);
        vin = (const C*)d.vdf;
    }
    const bool far = t.top <= L;
    if (far)
        for (int nu = L; nu >= t.top; nu--) launch_group_batched<T>(t, d, b, vin, d.up[nu], nrhs, s);
    mark(prof, 1, s);
    if (far) launch_group_batched<T>(t, d, b, vin, d.m2l, nrhs, s);
    mark(prof, 2, s);
    if (far)
        for (int nu = t.top; nu < L; nu++) launch_group_batched<T>(t, d, b, vin, d.down[nu], nrhs, s);
    mark(prof, 3, s);
    const C* nearp = (const C*)(sizeof(T) == 8 ? (const void*)d.neardf : (const void*)d.near32);
    const BsrDev* l2p = far ? &d.lv[L].down : nullptr;
    leaf_batched_kernel<T><<<(unsigned)nleaf, 256, 0, s>>>(
        nleaf, nrhs, d.nbr, nearp, vin, l2p ? l2p->rowptr : nullptr, l2p ? l2p->moff : nullptr, l2p ? l2p->rin : nullptr,
        l2p ? (const C*)(sizeof(T) == 8 ? l2p->mdf : l2p->m32) : nullptr, far ? d.lv[L].Ri : 0, far ? b.lc[L] : nullptr,
        (const double2*)v, d.potential ? nullptr : d.q, t.prm.kappa * t.prm.kappa, (double2*)out);
    CK(cudaGetLastError());
    mark(prof, 4, s);
}

size_t max_group_part(const OpsDev& d)
{
    size_t m = std::max({(size_t)d.m2l.nch * d.m2l.Pld, d.fz.plan[0].part, d.fz.plan[1].part});
    for (const Group& g : d.up) m = std::max(m, (size_t)g.nch * g.Pld);
    for (const Group& g : d.down) m = std::max(m, (size_t)g.nch * g.Pld);
    return m;
}

}  // namespace

void upload_ops(const Tree& t, OpsHost& h, OpsDev& d)
{
    const int L = t.L;
    d.lv.assign(L + 1, LevelDev());
    d.up.assign(L + 1, Group());
    d.down.assign(L + 1, Group());
    if (t.top <= L) {
        if (L - t.top + 1 > kMaxPass) fail(DAFMM_EBADARG, "too many far-field levels");
        std::vector<PassRef> m2l_passes;
        std::vector<const BsrHost*> m2l_hosts;
        std::vector<int> m2l_ldx;
        for (int nu = t.top; nu <= L; nu++) {
            d.lv[nu].Ri = h.lv[nu].Ri;
            d.lv[nu].Ro = h.lv[nu].Ro;
            build_group(d.up[nu], {PassRef{nu, 0}}, {&h.lv[nu].up}, {nu == L ? 16 : h.lv[nu + 1].Ro}, 0);
            if (nu < L) {
                // rows of level nu+1 that its M2L writes in every application
                const BsrHost& mc = h.lv[nu + 1].m2l;
                std::vector<char> init(mc.nrows, 0);
                for (int r = 0; r < mc.nrows; r++) init[r] = mc.rowptr[r + 1] > mc.rowptr[r];
                build_group(d.down[nu], {PassRef{nu, 2}}, {&h.lv[nu].down}, {h.lv[nu].Ri}, 1, &init);
            }
            m2l_passes.push_back(PassRef{nu, 1});
            m2l_hosts.push_back(&h.lv[nu].m2l);
            m2l_ldx.push_back(h.lv[nu].Ro);
        }
        build_group(d.m2l, m2l_passes, m2l_hosts, m2l_ldx, 0);
        CK(cudaFuncSetAttribute(stream_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, StreamCfg<float>::kCta));
        CK(cudaFuncSetAttribute(stream_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, StreamCfg<double>::kCta));
        CK(cudaFuncSetAttribute(leaf_apply_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kLeafPerCta * 17 * 2 * kLeafStageCols * (int)sizeof(float2)));
        CK(cudaFuncSetAttribute(leaf_apply_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kLeafPerCta * 17 * 2 * kLeafStageCols * (int)sizeof(double2)));
        d.fz.ctas[0] = fused_ctas<double>();
        d.fz.ctas[1] = fused_ctas<float>();
        // single right-hand side: the first up pass above the leaves reads the leaf
        // values through the P2M, the last L2L is applied with L2P by the leaf kernel
        BsrHost upc, leafc;
        const bool compose = t.top <= L - 1;
        if (compose) {
            upc = compose_up(h.lv[L - 1].up, h.lv[L].up);
            leafc = compose_leaf(h.lv[L - 1].down, h.lv[L].down);
        }
        build_fused(t, h, d, compose ? &upc : nullptr);
        d.fz.leaf_cmacs = 144.0 * t.N;
        for (int b = 0; b < h.lv[L].down.nrows; b++)
            for (int e = h.lv[L].down.rowptr[b]; e < h.lv[L].down.rowptr[b + 1]; e++) d.fz.leaf_cmacs += 16.0 * h.lv[L].down.rin[e];
        if (compose) {
            for (size_t e = 0; e < leafc.rin.size(); e++) d.fz.leaf_cmacs += 16.0 * leafc.rin[e];
            upload_bsr(upc, d.lv[L - 1].upc);
            upload_bsr(leafc, d.leafc);
        }
        // the leaf kernel stages its far-field blocks in shared memory when
        // every leaf has at most kLeafEnt composed blocks, one L2P block and
        // kLeafStageCols columns of each
        {
            const BsrHost& U = h.lv[L].down;
            int fcc = 0, fcl = 0;
            bool ok = t.top <= L;
            for (int b = 0; ok && b < U.nrows; b++) {
                const int ne = U.rowptr[b + 1] - U.rowptr[b];
                if (ne > 1) ok = false;
                if (ne == 1) fcl = std::max(fcl, U.rin[U.rowptr[b]]);
            }
            if (compose)
                for (int b = 0; ok && b < leafc.nrows; b++) {
                    int cols = 0;
                    for (int e = leafc.rowptr[b]; e < leafc.rowptr[b + 1]; e++) cols += leafc.rin[e];
                    if (leafc.rowptr[b + 1] - leafc.rowptr[b] > kLeafEnt) ok = false;
                    fcc = std::max(fcc, cols);
                }
            for (size_t e = 0; ok && e < U.moff.size(); e++) ok = U.moff[e] % 2 == 0;  // 16-byte aligned blocks
            if (compose)
                for (size_t e = 0; ok && e < leafc.moff.size(); e++) ok = leafc.moff[e] % 2 == 0;
            ok = ok && fcc <= kLeafStageCols && fcl <= kLeafStageCols && fcc + fcl > 0;
            d.fz.leaf_fcc = d.fz.leaf_fcc_plan = ok ? fcc : 0;
            d.fz.leaf_fcl = d.fz.leaf_fcl_plan = ok ? fcl : 0;
        }
        for (int nu = t.top; nu <= L; nu++) {
            // single-right-hand-side coefficients, zero once: rows no pass writes read as zero
            LevelDev& l = d.lv[nu];
            const size_t ns = (size_t)t.lv[nu].nslot();
            const size_t bytes[2] = {sizeof(double2), sizeof(float2)};
            for (int k = 0; k < 2; k++) {
                dev_alloc((char**)&l.fmp[k], bytes[k] * ns * std::max(l.Ro, 1));
                dev_alloc((char**)&l.flc[k], bytes[k] * ns * std::max(l.Ri, 1));
                dev_alloc((char**)&l.flcd[k], bytes[k] * ns * std::max(l.Ri, 1));
                CK(cudaMemset(l.fmp[k], 0, bytes[k] * ns * std::max(l.Ro, 1)));
                CK(cudaMemset(l.flc[k], 0, bytes[k] * ns * std::max(l.Ri, 1)));
                CK(cudaMemset(l.flcd[k], 0, bytes[k] * ns * std::max(l.Ri, 1)));
            }
        }
        for (int nu = t.top; nu <= L; nu++) {
            upload_bsr(h.lv[nu].up, d.lv[nu].up);
            upload_bsr(h.lv[nu].m2l, d.lv[nu].m2l);
            upload_bsr(h.lv[nu].down, d.lv[nu].down);
        }
    }
    // near blocks, transposed to [o][j][i]
    std::vector<double2> n64(9 * 256);
    std::vector<float2> n32(9 * 256);
    std::vector<float4> ndf(9 * 256);  // float pairs for the single-right-hand-side complex128 leaf kernel
    for (int o = 0; o < 9; o++)
        for (int i = 0; i < 16; i++)
            for (int j = 0; j < 16; j++) {
                cd v = h.near[o * 256 + i * 16 + j];
                n64[o * 256 + j * 16 + i] = make_double2(v.real(), v.imag());
                n32[o * 256 + j * 16 + i] = make_float2((float)v.real(), (float)v.imag());
                const float rh = (float)v.real(), ih = (float)v.imag();
                ndf[o * 256 + j * 16 + i] = make_float4(rh, ih, (float)(v.real() - (double)rh), (float)(v.imag() - (double)ih));
            }
    upload_vec(n64, &d.near64);
    upload_vec(n32, &d.near32);
    upload_vec(ndf, &d.neardf);
    // near-neighbour table of the leaves
    const int nleaf = t.nb * t.nb;
    std::vector<int> nbr((size_t)nleaf * 9, -1);
    for (int b = 0; b < nleaf; b++) {
        int bx = t.leaf_x[b], by = t.leaf_y[b];
        for (int sy = -1; sy <= 1; sy++)
            for (int sx = -1; sx <= 1; sx++) {
                int x = bx + sx, y = by + sy;
                if (x < 0 || y < 0 || x >= t.nb || y >= t.nb) continue;
                nbr[(size_t)b * 9 + (sy + 1) * 3 + (sx + 1)] = (int)morton_encode(x, y);
            }
    }
    upload_vec(nbr, &d.nbr);
    dev_alloc(&d.err, sizeof(int));
    CK(cudaMemset(d.err, 0, sizeof(int)));
    d.part_elems = max_group_part(d);
    ensure_scratch(t, d, 1);
}

void ensure_scratch(const Tree& t, OpsDev& d, int nrhs)
{
    if (nrhs <= d.nrhs_cap) return;
    const int L = t.L;
    for (int nu = t.top; nu <= L; nu++) {
        LevelDev& l = d.lv[nu];
        cudaFree(l.mp64);
        cudaFree(l.lc64);
        cudaFree(l.mp32);
        cudaFree(l.lc32);
        l.mp64 = l.lc64 = l.mp32 = l.lc32 = nullptr;
        const size_t ns = (size_t)t.lv[nu].nslot() * nrhs;
        dev_alloc((double2**)&l.mp64, sizeof(double2) * ns * l.Ro);
        dev_alloc((double2**)&l.lc64, sizeof(double2) * ns * l.Ri);
        dev_alloc((float2**)&l.mp32, sizeof(float2) * ns * l.Ro);
        dev_alloc((float2**)&l.lc32, sizeof(float2) * ns * l.Ri);
        CK(cudaMemset(l.mp64, 0, sizeof(double2) * ns * l.Ro));
        CK(cudaMemset(l.lc64, 0, sizeof(double2) * ns * l.Ri));
        CK(cudaMemset(l.mp32, 0, sizeof(float2) * ns * l.Ro));
        CK(cudaMemset(l.lc32, 0, sizeof(float2) * ns * l.Ri));
    }
    cudaFree(d.v32);
    d.v32 = nullptr;
    dev_alloc(&d.v32, sizeof(float2) * (size_t)t.N * nrhs);
    cudaFree(d.vdf);
    d.vdf = nullptr;
    dev_alloc(&d.vdf, sizeof(float4) * (size_t)t.N * nrhs);
    cudaFree(d.part);
    d.part = nullptr;
    dev_alloc((double2**)&d.part, sizeof(double2) * std::max<size_t>(d.part_elems, 1) * nrhs);
    d.nrhs_cap = nrhs;
    for (auto& row : d.gc)
        for (auto& G : row) {
            if (G.exec) cudaGraphExecDestroy(G.exec);
            if (G.graph) cudaGraphDestroy(G.graph);
            G = GraphCache();
        }
}

void set_batched_kernel(OpsDev& d, int mode)
{
    if (mode < 0 || mode > 2) fail(DAFMM_EBADARG, "batched kernel: 0 automatic, 1 CUDA cores, 2 tensor cores");
    if (mode == d.batched_kernel) return;
    d.batched_kernel = mode;
    // captured applications hold the previous kernels
    for (auto& row : d.gc)
        for (auto& G : row) {
            if (G.exec) cudaGraphExecDestroy(G.exec);
            if (G.graph) cudaGraphDestroy(G.graph);
            G = GraphCache();
        }
}

void set_leaf_staging(OpsDev& d, bool on)
{
    const int fcc = on ? d.fz.leaf_fcc_plan : 0, fcl = on ? d.fz.leaf_fcl_plan : 0;
    if (fcc == d.fz.leaf_fcc && fcl == d.fz.leaf_fcl) return;
    d.fz.leaf_fcc = fcc;
    d.fz.leaf_fcl = fcl;
    // captured applications hold the previous launch of the leaf kernel
    for (auto& row : d.gc)
        for (auto& G : row) {
            if (G.exec) cudaGraphExecDestroy(G.exec);
            if (G.graph) cudaGraphDestroy(G.graph);
            G = GraphCache();
        }
}

void set_batched_grid(OpsDev& d, int cps)
{
    if (cps < 0 || cps > 32) fail(DAFMM_EBADARG, "CTAs per SM must lie in 0..32");
    if (cps == d.batched_cps) return;
    d.batched_cps = cps;
    for (auto& row : d.gc)
        for (auto& G : row) {
            if (G.exec) cudaGraphExecDestroy(G.exec);
            if (G.graph) cudaGraphDestroy(G.graph);
            G = GraphCache();
        }
}

void profile_enable(OpsDev& d, bool on)
{
    d.profile = on;
    d.ev_used = 0;
    d.ev_fused.clear();
}

void profile_read(OpsDev& d, dafmm_profile_t& p)
{
    std::memset(&p, 0, sizeof(p));
    for (size_t c = 0; c + 5 <= d.ev_used; c += 5) {
        float ms[4];
        CK(cudaEventSynchronize(d.events[c + 4]));
        for (int k = 0; k < 4; k++) CK(cudaEventElapsedTime(&ms[k], d.events[c + k], d.events[c + k + 1]));
        if (!d.ev_fused[c / 5]) {
            p.ms_up += ms[0];
            p.ms_m2l += ms[1];
            p.ms_down += ms[2];
        }
        p.ms_far += ms[0] + ms[1] + ms[2];
        p.ms_leaf += ms[3];
        p.ms_total += ms[0] + ms[1] + ms[2] + ms[3];
        p.calls++;
    }
}

void free_ops(OpsDev& d)
{
    gmres_work_free(d.gw);
    gmres_many_free(d.gm);
    d.gm = nullptr;
    d.gw = nullptr;
    for (cudaEvent_t e : d.events) cudaEventDestroy(e);
    d.events.clear();
    for (auto& row : d.gc)
        for (auto& G : row) {
            if (G.exec) cudaGraphExecDestroy(G.exec);
            if (G.graph) cudaGraphDestroy(G.graph);
        }
    for (cudaEvent_t e : d.placeholder)
        if (e) cudaEventDestroy(e);
    if (d.cap_stream) cudaStreamDestroy(d.cap_stream);
    free_bsr(d.leafc);
    for (auto& l : d.lv) {
        free_bsr(l.up);
        free_bsr(l.m2l);
        free_bsr(l.down);
        free_bsr(l.upc);
        cudaFree(l.mp64);
        cudaFree(l.lc64);
        cudaFree(l.mp32);
        cudaFree(l.lc32);
        for (int k = 0; k < 2; k++) {
            cudaFree(l.fmp[k]);
            cudaFree(l.flc[k]);
            cudaFree(l.flcd[k]);
        }
    }
    free_fused(d.fz);
    for (auto& g : d.up) free_group(g);
    for (auto& g : d.down) free_group(g);
    free_group(d.m2l);
    d.lv.clear();
    cudaFree(d.near64);
    cudaFree(d.neardf);
    cudaFree(d.near32);
    cudaFree(d.nbr);
    cudaFree(d.q);
    cudaFree(d.v32);
    cudaFree(d.vdf);
    cudaFree(d.part);
    cudaFree(d.err);
    d = OpsDev();
}

int sync_and_check(OpsDev& d, cudaStream_t stream)
{
    CK(cudaStreamSynchronize(stream));
    if (!d.err) return DAFMM_OK;
    int flag = 0;
    CK(cudaMemcpy(&flag, d.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        // a warp that gave up may have left split-row counters armed
        auto rearm = [](Group& g) {
            if (g.cnt) CK(cudaMemset(g.cnt, 0, sizeof(int) * std::max(g.nch, 1)));
        };
        for (auto& g : d.up) rearm(g);
        for (auto& g : d.down) rearm(g);
        rearm(d.m2l);
        for (FusedPlan& P : d.fz.plan)
            if (P.cnt) CK(cudaMemset(P.cnt, 0, sizeof(int) * std::max(P.nch, 1)));
        if (d.fz.done) CK(cudaMemset(d.fz.done, 0, sizeof(int) * (kMaxPass + 1) * kDoneStride));
        CK(cudaMemset(d.err, 0, sizeof(int)));
        return DAFMM_ETIMEOUT;
    }
    return DAFMM_OK;
}

int launches_per_call(const Tree& t, const OpsDev& d, int precision)
{
    return 1 + (t.top <= t.L && d.fz.plan[precision == DAFMM_FP64 ? 0 : 1].nch > 0 ? 1 : 0);  // fused far field, leaf kernel
}

namespace {

// Take five fresh events from the handle's pool for one profiled call.
cudaEvent_t* next_profile_events(OpsDev& d)
{
    if (!d.profile || d.ev_used + 5 > (size_t)5 * 65536) return nullptr;
    while (d.events.size() < d.ev_used + 5) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        d.events.push_back(e);
    }
    d.ev_used += 5;
    d.ev_fused.resize(d.ev_used / 5, 0);
    return &d.events[d.ev_used - 5];
}

void run_eager(const Tree& t, OpsDev& d, const double* v, double* out, int nrhs, int precision, cudaStream_t stream, bool prof);

// Capture the application into the cache slot G (on the private stream),
// with event-record nodes at the five pass marks when `marks` (each node
// costs about 2.5 us of latency on the path, so only profiled calls carry them).
void capture(const Tree& t, OpsDev& d, const double* v, double* out, int nrhs, int precision, GraphCache& G, bool marks)
{
    if (!d.cap_stream) CK(cudaStreamCreateWithFlags(&d.cap_stream, cudaStreamNonBlocking));
    for (int k = 0; k < 5; k++)
        if (!d.placeholder[k]) CK(cudaEventCreate(&d.placeholder[k]));
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(d.cap_stream, cudaStreamCaptureModeThreadLocal));
    tl_capture_events = marks ? d.placeholder : nullptr;
    try {
        run_eager(t, d, v, out, nrhs, precision, d.cap_stream, false);
    } catch (...) {
        tl_capture_events = nullptr;
        cudaStreamEndCapture(d.cap_stream, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
    }
    tl_capture_events = nullptr;
    CK(cudaStreamEndCapture(d.cap_stream, &graph));
    if (G.exec) {
        // same topology, new pointers: update in place; the exec keeps the
        // node identities of the graph it was instantiated from
        cudaGraphExecUpdateResultInfo info;
        if (G.marks == marks && cudaGraphExecUpdate(G.exec, graph, &info) == cudaSuccess) {
            CK(cudaGraphDestroy(graph));
            G.v = v;
            G.out = out;
            G.nrhs = nrhs;
            return;
        }
        cudaGetLastError();
        cudaGraphExecDestroy(G.exec);
        cudaGraphDestroy(G.graph);
        G = GraphCache();
    }
    cudaError_t e = cudaGraphInstantiate(&G.exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(graph);
        G = GraphCache();
        fail(DAFMM_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    G.graph = graph;
    // locate the event-record nodes of the five marks
    size_t n = 0;
    CK(cudaGraphGetNodes(graph, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    CK(cudaGraphGetNodes(graph, nodes.data(), &n));
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType ty;
        CK(cudaGraphNodeGetType(nd, &ty));
        if (ty != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev;
        CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
        for (int k = 0; k < 5; k++)
            if (ev == d.placeholder[k]) G.ev_node[k] = nd;
    }
    G.v = v;
    G.out = out;
    G.nrhs = nrhs;
    G.marks = marks;
}

}  // namespace

void apply_potential(const Tree& t, OpsDev& d, int nrhs, const double* v, double* out, int precision, cudaStream_t stream)
{
    // the same passes with the leaf epilogue writing K v; launched directly (no graph)
    if (nrhs < 1 || nrhs > kMaxRhs) fail(DAFMM_EBADARG, "nrhs must lie in 1..64");
    if (t.L >= 64) fail(DAFMM_EBADARG, "tree too deep");
    cudaGetLastError();
    ensure_scratch(t, d, nrhs);
    d.potential = true;
    try {
        run_eager(t, d, v, out, nrhs, precision, stream, false);
    } catch (...) {
        d.potential = false;
        throw;
    }
    d.potential = false;
}

void apply_matvec(const Tree& t, OpsDev& d, int nrhs, const double* v, double* out, int precision, cudaStream_t stream)
{
    if (nrhs < 1 || nrhs > kMaxRhs) fail(DAFMM_EBADARG, "nrhs must lie in 1..64");
    if (t.L >= 64) fail(DAFMM_EBADARG, "tree too deep");
    cudaGetLastError();  // launch checks below must see only this call's errors
    ensure_scratch(t, d, nrhs);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(stream, &cs));
    if (d.stall_pass >= 0 && nrhs == 1 && cs == cudaStreamCaptureStatusNone) {
        // test support: this application only, launched directly
        try {
            run_eager(t, d, v, out, nrhs, precision, stream, false);
        } catch (...) {
            d.stall_pass = -1;
            throw;
        }
        d.stall_pass = -1;
        return;
    }
    if (cs != cudaStreamCaptureStatusNone) {
        // the caller is capturing: put the kernels into the caller's graph
        run_eager(t, d, v, out, nrhs, precision, stream, false);
        return;
    }
    // a cached graph for these pointers (with pass marks when profiling),
    // else the least recently used slot
    GraphCache* G = nullptr;
    for (auto& c : d.gc[precision])
        if (c.exec && c.v == v && c.out == out && c.nrhs == nrhs && c.marks == d.profile) G = &c;
    if (!G) {
        G = &d.gc[precision][0];
        for (auto& c : d.gc[precision])
            if (c.used < G->used) G = &c;
        capture(t, d, v, out, nrhs, precision, *G, d.profile);
    }
    G->used = ++d.gc_clock;
    if (d.profile) {
        cudaEvent_t* ev = next_profile_events(d);
        if (ev) d.ev_fused.back() = nrhs == 1;
        for (int k = 0; k < 5; k++) {
            cudaEvent_t e = ev ? ev[k] : d.placeholder[k];
            if (G->ev_node[k]) CK(cudaGraphExecEventRecordNodeSetEvent(G->exec, G->ev_node[k], e));
        }
    } else {
        for (int k = 0; k < 5; k++)
            if (G->ev_node[k]) CK(cudaGraphExecEventRecordNodeSetEvent(G->exec, G->ev_node[k], d.placeholder[k]));
    }
    CK(cudaGraphLaunch(G->exec, stream));
}

namespace {
void run_eager(const Tree& t, OpsDev& d, const double* v, double* out, int nrhs, int precision, cudaStream_t stream, bool prof)
{
    const int k = precision == DAFMM_FP64 ? 0 : 1;
    if (nrhs == 1) {
        auto fill = [&](auto& b) {
            using C = typename std::remove_pointer<decltype(b.part)>::type;
            for (int nu = t.top; nu <= t.L; nu++) {
                b.mp[nu] = (C*)d.lv[nu].fmp[k];
                b.lc[nu] = (C*)d.lv[nu].flc[k];
                b.lcd[nu] = (C*)d.lv[nu].flcd[k];
            }
            b.part = (C*)d.part;
        };
        if (k == 0) {
            FBufs<double> b;
            fill(b);
            run_fused<double>(t, d, b, v, out, stream, prof ? &d : nullptr);
        } else {
            FBufs<float> b;
            fill(b);
            run_fused<float>(t, d, b, v, out, stream, prof ? &d : nullptr);
        }
        return;
    }
    if (k == 0) {
        Bufs<double> b;
        for (int nu = t.top; nu <= t.L; nu++) {
            b.mp[nu] = (double2*)d.lv[nu].mp64;
            b.lc[nu] = (double2*)d.lv[nu].lc64;
        }
        b.part = (double2*)d.part;
        run_batched<double>(t, d, b, d.v32, v, out, nrhs, stream, prof ? &d : nullptr);
    } else {
        Bufs<float> b;
        for (int nu = t.top; nu <= t.L; nu++) {
            b.mp[nu] = (float2*)d.lv[nu].mp32;
            b.lc[nu] = (float2*)d.lv[nu].lc32;
        }
        b.part = (float2*)d.part;
        run_batched<float>(t, d, b, d.v32, v, out, nrhs, stream, prof ? &d : nullptr);
    }
}
}  // namespace

// ---------------------------------------------------------------------------
// Allocation-free application.  Some callers cannot let the library allocate
// device memory at call time: processes whose device memory is owned by their
// own pool (a cudaMalloc there can fail or fragment the pool), hot loops that
// cannot afford cudaMalloc's implicit device synchronisation, and deployments
// that must fix all memory before they start.  For them the scratch of one
// single-RHS application (chunk partials, and per level the multipoles, the
// locals written by M2L and the locals written by the parent's L2L) lives in
// this fixed device array instead of the handle's
// grow-on-demand buffers.  Every GPU that loads the library holds the array
// until the process exits; all calls on a device share it, so calls whose
// kernels overlap in time on that device race.
namespace {

constexpr int kMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[DAFMM_NOALLOC_SCRATCH_BYTES];
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the static scratch on the current device.  The first call
// on a device resolves it with cudaGetSymbolAddress (this set-up should happen
// before any stream capture); later calls reuse the cached address.
unsigned char* noalloc_scratch()
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) fail(DAFMM_EBADARG, "device ordinal out of range for the static scratch");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            fail(DAFMM_ECUDA, std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    return (unsigned char*)g_noalloc_addr[dev];
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

template <typename T>
void run_noalloc(const Tree& t, const OpsDev& d, const double* v, double* out, cudaStream_t s)
{
    using C = typename V2<T>::t;
    const int L = t.L;
    const bool far = t.top <= L;
    if (L >= 64) fail(DAFMM_EBADARG, "tree too deep for the allocation-free path");
    // layout: chunk partials, then per level multipoles, locals from M2L and locals from the parent
    size_t need = align256(sizeof(C) * std::max<size_t>(d.part_elems, 1));
    if (far)
        for (int nu = t.top; nu <= L; nu++)
            need += align256(sizeof(C) * (size_t)t.lv[nu].nslot() * std::max(d.lv[nu].Ro, 1)) +
                    2 * align256(sizeof(C) * (size_t)t.lv[nu].nslot() * std::max(d.lv[nu].Ri, 1));
    if (need > (size_t)DAFMM_NOALLOC_SCRATCH_BYTES)
        fail(DAFMM_EBADARG, "problem needs " + std::to_string(need) + " bytes of scratch; the allocation-free path holds " +
                                std::to_string((size_t)DAFMM_NOALLOC_SCRATCH_BYTES) + " (use dafmm_matvec)");
    unsigned char* base = noalloc_scratch();
    // the array keeps the previous call's contents: start from zeros
    CK(cudaMemsetAsync(base, 0, need, s));
    size_t off = 0;
    FBufs<T> b;
    b.part = (C*)(base + off);
    off += align256(sizeof(C) * std::max<size_t>(d.part_elems, 1));
    if (far)
        for (int nu = t.top; nu <= L; nu++) {
            b.mp[nu] = (C*)(base + off);
            // at least one row per slot even at rank 0, as in the handle's own buffers
            off += align256(sizeof(C) * (size_t)t.lv[nu].nslot() * std::max(d.lv[nu].Ro, 1));
            b.lc[nu] = (C*)(base + off);
            off += align256(sizeof(C) * (size_t)t.lv[nu].nslot() * std::max(d.lv[nu].Ri, 1));
            b.lcd[nu] = (C*)(base + off);
            off += align256(sizeof(C) * (size_t)t.lv[nu].nslot() * std::max(d.lv[nu].Ri, 1));
        }
    run_fused<T>(t, d, b, v, out, s, nullptr);
}

}  // namespace

void apply_matvec_noalloc(const Tree& t, const OpsDev& d, const double* v, double* out, int precision, cudaStream_t stream)
{
    cudaGetLastError();  // launch checks below must see only this call's errors
    if (precision == DAFMM_FP64)
        run_noalloc<double>(t, d, v, out, stream);
    else
        run_noalloc<float>(t, d, v, out, stream);
}

}  // namespace dafmm
