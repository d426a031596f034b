// HODLR approximation of A (Ambikasaran & Darve; the preconditioner of the
// Hybrid solver, Section 6, Eq. hybrid) and its application on the device.
//
// The index set (Morton order, so every range is a spatially compact block of
// leaves) is halved recursively down to leaves of n_leaf unknowns.  At a node
// with halves I1, I2 the off-diagonal blocks are compressed by partially
// pivoted ACA to a fixed rank r (or to a tolerance): A(I1,I2) ~ U12 V12,
// A(I2,I1) ~ U21 V21.  Then, with D = diag(A1~, A2~) the children's
// approximations,
//     A~ = D + Ubar W,  Ubar = diag(U12, U21),  W = [[0, V12], [V21, 0]],
//     A~^{-1} = D^{-1} - Ut S^{-1} W D^{-1},  Ut = D^{-1} Ubar,  S = I + W Ut
// (Sherman-Morrison-Woodbury).  The factorisation (host, FP64, bottom-up)
// inverts the dense leaf blocks and forms Ut and S^{-1} at every node; the
// apply (device) multiplies the leaf inverses, then per level from the
// leaves up computes t = W x (segmented reductions), s = S^{-1} t and
// x -= Ut s.  Apply cost O(r N log N) (Section 6.1).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

#include "aca.h"
#include "ops.h"

namespace dafmm {
namespace {

#define CK(x)                                                                                     \
    do {                                                                                          \
        cudaError_t e_ = (x);                                                                     \
        if (e_ != cudaSuccess) {                                                                  \
            cudaGetLastError();                                                                   \
            fail(DAFMM_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_));                   \
        }                                                                                         \
    } while (0)

// Dense complex inverse by Gauss-Jordan with partial pivoting (row-major n x n).
bool invert(std::vector<cd>& a, int n)
{
    std::vector<cd> inv((size_t)n * n, cd(0));
    for (int i = 0; i < n; i++) inv[(size_t)i * n + i] = 1.0;
    for (int c = 0; c < n; c++) {
        int p = c;
        double b = std::abs(a[(size_t)c * n + c]);
        for (int r = c + 1; r < n; r++)
            if (std::abs(a[(size_t)r * n + c]) > b) {
                b = std::abs(a[(size_t)r * n + c]);
                p = r;
            }
        if (b == 0.0) return false;
        if (p != c)
            for (int k = 0; k < n; k++) {
                std::swap(a[(size_t)c * n + k], a[(size_t)p * n + k]);
                std::swap(inv[(size_t)c * n + k], inv[(size_t)p * n + k]);
            }
        const cd d = 1.0 / a[(size_t)c * n + c];
        for (int k = 0; k < n; k++) {
            a[(size_t)c * n + k] *= d;
            inv[(size_t)c * n + k] *= d;
        }
        for (int r = 0; r < n; r++) {
            if (r == c) continue;
            const cd f = a[(size_t)r * n + c];
            if (f == cd(0)) continue;
            for (int k = 0; k < n; k++) {
                a[(size_t)r * n + k] -= f * a[(size_t)c * n + k];
                inv[(size_t)r * n + k] -= f * inv[(size_t)c * n + k];
            }
        }
    }
    a.swap(inv);
    return true;
}

}  // namespace

// Host factors.  Level l = 0..H-1 holds the internal nodes of size N >> l.
struct HodlrLevelHost {
    int r = 0;             // rank (padded over the level's nodes with zero columns)
    std::vector<cd> R;     // r x N: row factors, R[q][i] = V21[q][i] for i in I1, V12[q][i] for i in I2
    std::vector<cd> Ut;    // N x r: Ut[i][q] = (A1~^{-1} U12)[i][q] for i in I1, (A2~^{-1} U21) for I2
    std::vector<cd> Sinv;  // per node (2r x 2r, row-major)
    std::vector<cd> U;     // N x r: the uncorrected U12 / U21 (kept for the dense export)
};

constexpr int kHodlrMaxLevels = 24;  // levels of the apply launch

struct HodlrDevLevel {
    int r = 0;
    double2 *R64 = nullptr, *Ut64 = nullptr, *S64 = nullptr;  // float pairs (see to_pairs)
    float2 *R32 = nullptr, *Ut32 = nullptr, *S32 = nullptr;
};

}  // namespace dafmm

struct dafmm_hodlr {
    const dafmm_tree* tree = nullptr;
    long N = 0;
    int leaf = 64, H = 0;
    std::vector<dafmm::cd> leafA;    // nleaf x leaf x leaf dense blocks (row-major), for the export
    std::vector<dafmm::cd> leafInv;  // their inverses
    std::vector<dafmm::HodlrLevelHost> lv;
    // device
    double2* inv64 = nullptr;  // float pairs (see to_pairs)
    float2* inv32 = nullptr;
    std::vector<dafmm::HodlrDevLevel> dlv;
    void* t_part = nullptr;  // partial sums of W x (complex128 size): rmax x N / leaf
    void* s_buf = nullptr;   // s per node, two parity halves of 2 rmax x N / leaf
    void* xw = nullptr;      // complex64 work vector (mixed precision)
    long sbuf_half = 0;      // entries of one parity half of s_buf
    unsigned* bar = nullptr;  // grid barrier: arrivals, exits
    int* err = nullptr;       // set when a wait of the apply gave up
    int ncta = 1;             // CTAs of the apply launch
    int ncta_default = 1;     // the width chosen at build
    long ncta_cap = 1;        // CTAs resident at once
    mutable int stall = 0;    // test support: the next apply waits for one CTA too many
    int rmax = 0;
    double seconds = 0;
    // several right-hand sides (hodlr_solve with nrhs > 1), grown on demand:
    // work vector [N][nrhs], segment partials [segment][q][nrhs], s per node [node][2 r][nrhs]
    void* bx = nullptr;
    void* bpart = nullptr;
    void* bs = nullptr;
    int bcap = 0;  // right-hand sides the buffers hold
};

namespace dafmm {
namespace {

// Apply the host factors of the subtree (level l, node k) to the columns
// cols[c] (each the node's n unknowns), in place: x = A~^{-1} b.
void host_solve(const dafmm_hodlr& h, int l, long k, std::vector<std::vector<cd>>& cols)
{
    const long n = h.N >> l;
    if (l == h.H) {
        const cd* inv = &h.leafInv[(size_t)k * h.leaf * h.leaf];
        std::vector<cd> tmp(h.leaf);
        for (auto& b : cols) {
            for (int i = 0; i < h.leaf; i++) {
                cd s = 0;
                for (int j = 0; j < h.leaf; j++) s += inv[(size_t)i * h.leaf + j] * b[j];
                tmp[i] = s;
            }
            std::copy(tmp.begin(), tmp.end(), b.begin());
        }
        return;
    }
    const long half = n / 2;
    std::vector<std::vector<cd>> c1(cols.size()), c2(cols.size());
    for (size_t c = 0; c < cols.size(); c++) {
        c1[c].assign(cols[c].begin(), cols[c].begin() + half);
        c2[c].assign(cols[c].begin() + half, cols[c].end());
    }
    host_solve(h, l + 1, 2 * k, c1);
    host_solve(h, l + 1, 2 * k + 1, c2);
    const HodlrLevelHost& L = h.lv[l];
    const int r = L.r;
    const long i0 = k * n;
    const cd* S = &L.Sinv[(size_t)k * 4 * r * r];
    std::vector<cd> t(2 * r), s(2 * r);
    for (size_t c = 0; c < cols.size(); c++) {
        for (int q = 0; q < r; q++) {
            cd a = 0, b = 0;
            for (long i = 0; i < half; i++) a += L.R[(size_t)q * h.N + i0 + half + i] * c2[c][i];  // V12 x2
            for (long i = 0; i < half; i++) b += L.R[(size_t)q * h.N + i0 + i] * c1[c][i];         // V21 x1
            t[q] = a;
            t[r + q] = b;
        }
        for (int a = 0; a < 2 * r; a++) {
            cd v = 0;
            for (int b = 0; b < 2 * r; b++) v += S[(size_t)a * 2 * r + b] * t[b];
            s[a] = v;
        }
        for (long i = 0; i < half; i++) {
            cd v1 = c1[c][i], v2 = c2[c][i];
            for (int q = 0; q < r; q++) {
                v1 -= L.Ut[(size_t)(i0 + i) * r + q] * s[q];
                v2 -= L.Ut[(size_t)(i0 + half + i) * r + q] * s[r + q];
            }
            cols[c][i] = v1;
            cols[c][half + i] = v2;
        }
    }
}

template <typename V>
void up(const std::vector<V>& h, V** d)
{
    if (h.empty()) return;
    if (cudaMalloc((void**)d, sizeof(V) * h.size()) != cudaSuccess) {
        cudaGetLastError();
        fail(DAFMM_ENOMEM, "device allocation for the HODLR factors failed");
    }
    CK(cudaMemcpy(*d, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice));
}

// complex128 factors as float pairs {re hi, im hi, re lo, im lo} in the 16
// bytes of a double2 (hi the nearest float, lo the nearest float of the rest)
std::vector<double2> to_pairs(const std::vector<cd>& v)
{
    std::vector<double2> o(v.size());
    for (size_t k = 0; k < v.size(); k++) {
        const double re = v[k].real(), im = v[k].imag();
        const float rh = (float)re, ih = (float)im;
        const float f[4] = {rh, ih, (float)(re - (double)rh), (float)(im - (double)ih)};
        std::memcpy(&o[k], f, sizeof(f));
    }
    return o;
}
std::vector<float2> to32(const std::vector<cd>& v)
{
    std::vector<float2> o(v.size());
    for (size_t k = 0; k < v.size(); k++) o[k] = make_float2((float)v[k].real(), (float)v[k].imag());
    return o;
}

// ------------------------------------------------------------ kernels ----

template <typename T>
struct C2;
template <>
struct C2<double> {
    using t = double2;
};
template <>
struct C2<float> {
    using t = float2;
};

template <typename C>
__device__ __forceinline__ C cmul(C a, C b)
{
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// ------------------------------------------------------------------------
// The application x = A~^{-1} b is one cooperative launch.  CTA c owns the
// unknowns [c E, (c + 1) E) (E a power of two, a multiple of the leaf size):
//   1. x = D^{-1} b on its leaves;
//   then for every level l from the leaves up (n = N >> l, halves of h = n/2):
//   2. partial sums of t = W x over its segments (min(E, h) unknowns each);
//   3. each segment's share of s = S^{-1} t (S^{-1} t is linear in t, and a
//      segment adds to one half of t): the half's columns of S^{-1} times
//      the segment's partial sums;
//   4. grid barrier (every share is written; not needed at levels whose
//      nodes each lie in one CTA);
//   5. s of each segment's half as the sum of its node's shares (a fixed
//      order, so results do not depend on timing), then x -= Ut s on its
//      unknowns.
// Steps 5 and 2 of the next level touch only the CTA's own unknowns, so one
// barrier per level suffices.  Every wait has a time limit, after which the
// launch sets the handle's error flag and returns.

constexpr int kHT = 256;                              // threads per CTA
constexpr unsigned long long kHWaitNs = 200000000ull;  // 0.2 s per barrier

template <typename T>
struct HArgs {
    using C = typename C2<T>::t;
    long N;
    int H, lf, ncta, extra;
    long E;
    const C* inv;        // leaf inverses, column-major lf x lf per leaf
    const double2* b;    // right-hand side (complex128)
    double2* xout;       // result (complex128)
    C* x;                // work vector (xout itself in complex128)
    C* part;             // partial sums, [q][segment]
    C* sbuf;             // shares of s per segment, two buffers by level parity: [parity][segment][2 r]
    long sbuf_half;      // entries per parity buffer
    unsigned* bar;       // [0] barrier arrivals, [1] exits
    int* err;
    const C* R[kHodlrMaxLevels];  // r x N
    const C* U[kHodlrMaxLevels];  // Ut transposed: r x N
    const C* S[kHodlrMaxLevels];  // per node 2r x 2r row-major
    int r[kHodlrMaxLevels];
};

__device__ __forceinline__ unsigned long long h_clock()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned h_ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier: arrive, then wait until target arrivals (with a time and an
// iteration limit).  False, with *err set, when the wait gave up.
__device__ bool h_barrier(unsigned* arrive, unsigned target, int* err)
{
    __threadfence();
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        atomicAdd(arrive, 1u);
        const unsigned long long t0 = h_clock();
        for (unsigned it = 0; h_ld_acquire(arrive) < target; it++) {
            if (it > (1u << 24) || h_clock() - t0 > kHWaitNs) {
                atomicExch(err, 1);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;
}

// Bring [p, p + bytes) into L2 (16-byte aligned, a multiple of 16 bytes).
__device__ __forceinline__ void l2_prefetch(const void* p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Arithmetic of the apply.  complex64 (mixed precision): float2 values, FP32
// sums.  complex128: float pairs {re hi, im hi, re lo, im lo} in the 16 bytes
// of a double2 (double-float arithmetic, about 48 significant bits: FP64
// instructions issue at 1/64 of the FP32 rate on GB300), the factors stored
// so, the input split and the result rounded to double once.
__device__ __forceinline__ float4 as_f4(double2 d)
{
    union {
        double2 d;
        float4 f;
    } u;
    u.d = d;
    return u.f;
}
__device__ __forceinline__ double2 as_d2(float4 f)
{
    union {
        double2 d;
        float4 f;
    } u;
    u.f = f;
    return u.d;
}

// (sh, sl) += a b for float pairs: the product's rounding error by FMA, the
// cross terms, a two-sum into sh (explicitly rounded steps, never contracted).
__device__ __forceinline__ void pf_mac(float& sh, float& sl, float ah, float al, float bh, float bl)
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

// (h, l) = a + b for float pairs, renormalised.
__device__ __forceinline__ void pf_add(float& h, float& l, float ah, float al, float bh, float bl)
{
    const float s = __fadd_rn(ah, bh);
    const float v = __fsub_rn(s, ah);
    const float e = __fadd_rn(__fadd_rn(__fsub_rn(ah, __fsub_rn(s, v)), __fsub_rn(bh, v)), __fadd_rn(al, bl));
    h = __fadd_rn(s, e);
    l = __fsub_rn(e, __fsub_rn(h, s));
}

template <typename T>
struct Ar;

template <>
struct Ar<float> {
    using C = float2;
    struct A {
        float r, i;
    };
    static __device__ __forceinline__ A zero() { return A{0.f, 0.f}; }
    static __device__ __forceinline__ void mac(A& a, C m, C v)
    {
        a.r = fmaf(m.x, v.x, fmaf(-m.y, v.y, a.r));
        a.i = fmaf(m.x, v.y, fmaf(m.y, v.x, a.i));
    }
    static __device__ __forceinline__ void add(A& a, A b)
    {
        a.r += b.r;
        a.i += b.i;
    }
    static __device__ __forceinline__ void add_c(A& a, C v)
    {
        a.r += v.x;
        a.i += v.y;
    }
    static __device__ __forceinline__ A shfl_xor(A a, int o)
    {
        return A{__shfl_xor_sync(0xffffffffu, a.r, o), __shfl_xor_sync(0xffffffffu, a.i, o)};
    }
    static __device__ __forceinline__ C to_c(A a) { return make_float2(a.r, a.i); }
    static __device__ __forceinline__ C sub(C x, A a) { return make_float2(x.x - a.r, x.y - a.i); }
    static __device__ __forceinline__ C from64(double2 b) { return make_float2((float)b.x, (float)b.y); }
    static __device__ __forceinline__ double2 to64(C x) { return make_double2(x.x, x.y); }
};

template <>
struct Ar<double> {
    using C = double2;  // holds a float pair
    struct A {
        float rh, rl, ih, il;
    };
    static __device__ __forceinline__ A zero() { return A{0.f, 0.f, 0.f, 0.f}; }
    static __device__ __forceinline__ void mac(A& a, C mc, C vc)
    {
        const float4 m = as_f4(mc), v = as_f4(vc);
        pf_mac(a.rh, a.rl, m.x, m.z, v.x, v.z);
        pf_mac(a.rh, a.rl, -m.y, -m.w, v.y, v.w);
        pf_mac(a.ih, a.il, m.x, m.z, v.y, v.w);
        pf_mac(a.ih, a.il, m.y, m.w, v.x, v.z);
    }
    static __device__ __forceinline__ void add(A& a, A b)
    {
        pf_add(a.rh, a.rl, a.rh, a.rl, b.rh, b.rl);
        pf_add(a.ih, a.il, a.ih, a.il, b.ih, b.il);
    }
    static __device__ __forceinline__ void add_c(A& a, C vc)
    {
        const float4 v = as_f4(vc);
        pf_add(a.rh, a.rl, a.rh, a.rl, v.x, v.z);
        pf_add(a.ih, a.il, a.ih, a.il, v.y, v.w);
    }
    static __device__ __forceinline__ A shfl_xor(A a, int o)
    {
        return A{__shfl_xor_sync(0xffffffffu, a.rh, o), __shfl_xor_sync(0xffffffffu, a.rl, o), __shfl_xor_sync(0xffffffffu, a.ih, o),
                 __shfl_xor_sync(0xffffffffu, a.il, o)};
    }
    static __device__ __forceinline__ C to_c(A a) { return as_d2(make_float4(a.rh, a.ih, a.rl, a.il)); }
    static __device__ __forceinline__ C sub(C xc, A a)
    {
        const float4 x = as_f4(xc);
        float rh, rl, ih, il;
        pf_add(rh, rl, x.x, x.z, -a.rh, -a.rl);
        pf_add(ih, il, x.y, x.w, -a.ih, -a.il);
        return as_d2(make_float4(rh, ih, rl, il));
    }
    static __device__ __forceinline__ C from64(double2 b)
    {
        const float rh = __double2float_rn(b.x), ih = __double2float_rn(b.y);
        return as_d2(make_float4(rh, ih, __double2float_rn(b.x - (double)rh), __double2float_rn(b.y - (double)ih)));
    }
    static __device__ __forceinline__ double2 to64(C xc)
    {
        const float4 x = as_f4(xc);
        return make_double2((double)x.x + (double)x.z, (double)x.y + (double)x.w);
    }
};

// This CTA's columns [e0, e0 + E) of R and Ut of level l to L2.
template <typename T>
__device__ __forceinline__ void prefetch_rows(const HArgs<T>& a, int l, long e0, int tid)
{
    using C = typename C2<T>::t;
    if (l < 0) return;
    const int r = a.r[l];
    for (int k = tid; k < 2 * r; k += kHT) {
        const C* base = k < r ? a.R[l] + (size_t)k * a.N : a.U[l] + (size_t)(k - r) * a.N;
        for (long o = 0; o < a.E; o += 2048) l2_prefetch(base + e0 + o, (unsigned)(min(a.E - o, 2048L) * sizeof(C)));
    }
}

template <typename T>
__global__ void __launch_bounds__(kHT, 2) hodlr_apply_kernel(const __grid_constant__ HArgs<T> a)
{
    using C = typename C2<T>::t;
    using P = Ar<T>;
    using A = typename P::A;
    extern __shared__ __align__(16) unsigned char hsm[];
    C* sh = (C*)hsm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kW = kHT / 32;
    const long E = a.E, e0 = (long)blockIdx.x * E;
    const int lf = a.lf;
    // factors to L2 ahead of use: a 1/ncta slice of every level's S blocks
    // now, this CTA's columns of R and Ut one level ahead (prefetch_rows)
    prefetch_rows(a, a.H - 1, e0, tid);
    for (int l = a.H - 1; l >= 0; l--) {
        const int r = a.r[l];
        if (tid == 0 && r > 0) {
            const size_t sb = (size_t)(1L << l) * 4 * r * r * sizeof(C);
            const size_t sl = (sb / a.ncta + 15) / 16 * 16, b0 = (size_t)blockIdx.x * sl;
            for (size_t o = b0; o < min(sb, b0 + sl); o += 32768)
                l2_prefetch((const char*)a.S[l] + o, (unsigned)min((size_t)32768, min(sb, b0 + sl) - o));
        }
    }
    // 1. leaf inverses, `per` unknowns (whole leaves) staged at a time, so that x may alias b
    const long per = min(E, (long)max(lf, kHT));
    for (long g0 = e0; g0 < e0 + E; g0 += per) {
        __syncthreads();
        for (long k = tid; k < per; k += kHT) sh[k] = P::from64(a.b[g0 + k]);
        __syncthreads();
        for (long k = tid; k < per; k += kHT) {
            const long li = k / lf * lf, i = k - li;
            const C* M = a.inv + (size_t)((g0 + li) / lf) * lf * lf + i;
            A acc = P::zero();
            for (int j = 0; j < lf; j++) P::mac(acc, M[(size_t)j * lf], sh[li + j]);
            a.x[g0 + k] = P::to_c(acc);
        }
    }
    bool ok = true;
    unsigned nb = 0;
    for (int l = a.H - 1; l >= 0; l--) {
        const int r = a.r[l];
        if (r == 0) continue;
        const long n = a.N >> l, h = n >> 1;
        const long m = min(E, h), nslots = a.N / m;
        const C* R = a.R[l];
        prefetch_rows(a, l - 1, e0, tid);
        __syncthreads();  // this CTA's x is final for the level
        // 2. partials of W x: part[q][segment] over each of this CTA's segments
        // (four rows q of R per warp at a time, so that their loads overlap)
        for (long s0 = e0; s0 < e0 + E; s0 += m) {
            for (int q0 = warp; q0 < r; q0 += 4 * kW) {
                A acc[4] = {P::zero(), P::zero(), P::zero(), P::zero()};
                for (long i = s0 + lane; i < s0 + m; i += 32) {
                    const C xv = a.x[i];
#pragma unroll
                    for (int u = 0; u < 4; u++)
                        if (q0 + u * kW < r) P::mac(acc[u], R[(size_t)(q0 + u * kW) * a.N + i], xv);
                }
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int u = 0; u < 4; u++) P::add(acc[u], P::shfl_xor(acc[u], o));
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (lane == u && q0 + u * kW < r) a.part[(size_t)(q0 + u * kW) * nslots + s0 / m] = P::to_c(acc[u]);
            }
        }
        __syncthreads();  // this CTA's partials are written
        // 3. each segment's share of s = S^{-1} t: t takes half 2's sums in rows [0, r) and
        //    half 1's in [r, 2r), so segment g of half hh adds S[:, cols] part_g with cols
        //    [0, r) (hh = 1) or [r, 2r) (hh = 0).  Rows of S are split over p consecutive lanes.
        const int R2 = 2 * r;
        C* cb = a.sbuf + (size_t)(l & 1) * a.sbuf_half;  // shares: [segment][2 r]
        int p = 1;
        while (p < 32 && 2 * p * R2 <= kHT) p *= 2;
        const int rpp = kHT / p, npass = (R2 + rpp - 1) / rpp, piece = tid % p;
        for (long s0 = e0; s0 < e0 + E; s0 += m) {
            const long g = s0 / m, nd = s0 / n;
            const int colb = (s0 - nd * n) >= h ? 0 : r;
            for (int q = tid; q < r; q += kHT) sh[q] = a.part[(size_t)q * nslots + g];
            __syncthreads();
            const C* Sn = a.S[l] + (size_t)nd * 4 * r * r + colb;
            const int cols = (r + p - 1) / p;
            for (int pass = 0; pass < npass; pass++) {
                const int aa = pass * rpp + tid / p;
                A acc = P::zero();
                if (aa < R2) {
                    const C* row = Sn + (size_t)aa * R2;
                    const int b1 = min(r, (piece + 1) * cols);
#pragma unroll 8
                    for (int bb = piece * cols; bb < b1; bb++) P::mac(acc, row[bb], sh[bb]);
                }
                for (int o = p / 2; o > 0; o >>= 1) P::add(acc, P::shfl_xor(acc, o));
                if (aa < R2 && piece == 0) cb[(size_t)g * R2 + aa] = P::to_c(acc);
            }
            __syncthreads();
        }
        // 4. every share is written; a level whose nodes each lie in one CTA reads only its own
        if (E < n) {
            nb++;
            if (!h_barrier(&a.bar[0], nb * (unsigned)a.ncta + (unsigned)a.extra, a.err)) {
                ok = false;
                break;
            }
        } else {
            __threadfence_block();
            __syncthreads();
        }
        // 5. per segment: s of its half = the sum of the node's shares (a fixed order: rows q
        //    over p2 lanes, each lane its strided subset, then a shuffle tree), staged in shared
        //    memory; then x -= Ut s on the segment, the sum over q split between tpe threads
        //    per unknown when the segment is shorter than the CTA
        const C* U = a.U[l];
        const int tpe = m >= kHT ? 1 : (int)(kHT / m);
        C* red = sh + 2 * r;  // tpe x m partial sums (tpe > 1)
        int p2 = 1;
        while (p2 < 32 && 2 * p2 * r <= kHT) p2 *= 2;
        const int rpp2 = kHT / p2, npass2 = (r + rpp2 - 1) / rpp2, piece2 = tid % p2;
        for (long s0 = e0; s0 < e0 + E; s0 += m) {
            const long nd = s0 / n;
            const int hoff = (s0 - nd * n) >= h ? r : 0;
            const long ga = nd * n / m, gn = n / m;  // the node's segments [ga, ga + gn)
            __syncthreads();
            for (int pass = 0; pass < npass2; pass++) {
                const int q = pass * rpp2 + tid / p2;
                A acc = P::zero();
                if (q < r) {
                    const C* Pq = cb + (size_t)ga * R2 + hoff + q;
#pragma unroll 8
                    for (long k = piece2; k < gn; k += p2) P::add_c(acc, __ldcg(Pq + (size_t)k * R2));
                }
                for (int o = p2 / 2; o > 0; o >>= 1) P::add(acc, P::shfl_xor(acc, o));
                if (q < r && piece2 == 0) sh[q] = P::to_c(acc);
            }
            __syncthreads();
            const int g = tid / (int)min(m, (long)kHT);
            for (long k = tid % min(m, (long)kHT); k < m; k += min(m, (long)kHT)) {
                const long i = s0 + k;
                A acc = P::zero();
                int q = g;
                for (; q + 7 * tpe < r; q += 8 * tpe) {
                    C u[8];
#pragma unroll
                    for (int v = 0; v < 8; v++) u[v] = U[(size_t)(q + v * tpe) * a.N + i];
#pragma unroll
                    for (int v = 0; v < 8; v++) P::mac(acc, u[v], sh[q + v * tpe]);
                }
                for (; q < r; q += tpe) P::mac(acc, U[(size_t)q * a.N + i], sh[q]);
                if (tpe == 1)
                    a.x[i] = P::sub(a.x[i], acc);
                else
                    red[(size_t)g * m + k] = P::to_c(acc);
            }
            if (tpe > 1) {
                __syncthreads();
                for (long k = tid; k < m; k += kHT) {
                    A acc = P::zero();
                    for (int gg = 0; gg < tpe; gg++) P::add_c(acc, red[(size_t)gg * m + k]);
                    a.x[s0 + k] = P::sub(a.x[s0 + k], acc);
                }
            }
        }
    }
    // the result in complex128 (in place for complex128: each thread its own unknowns)
    if (ok)
        for (long i = e0 + tid; i < e0 + E; i += kHT) a.xout[i] = P::to64(a.x[i]);
    // the last CTA to leave re-arms the barrier for the next launch
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&a.bar[1], 1u) == (unsigned)a.ncta - 1) {
            a.bar[0] = 0;
            a.bar[1] = 0;
            __threadfence();
        }
    }
}

template <typename T>
size_t apply_smem(const dafmm_hodlr& h)
{
    using C = typename C2<T>::t;
    return sizeof(C) * (size_t)std::max<long>(std::max(h.leaf, kHT), 2L * std::max(h.rmax, 1) + kHT);
}

template <typename T>
void apply(const dafmm_hodlr& h, const double2* b, double2* xout, cudaStream_t s)
{
    using C = typename C2<T>::t;
    HArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.N = h.N;
    a.H = h.H;
    a.lf = h.leaf;
    a.ncta = h.ncta;
    a.E = h.N / h.ncta;
    a.extra = h.stall ? 1 : 0;
    h.stall = 0;
    a.inv = (const C*)(sizeof(T) == 8 ? (const void*)h.inv64 : (const void*)h.inv32);
    a.b = b;
    a.xout = xout;
    a.x = sizeof(T) == 8 ? (C*)xout : (C*)h.xw;
    a.part = (C*)h.t_part;
    a.sbuf = (C*)h.s_buf;
    a.sbuf_half = h.sbuf_half;
    a.bar = h.bar;
    a.err = h.err;
    for (int l = 0; l < h.H; l++) {
        const HodlrDevLevel& L = h.dlv[l];
        a.r[l] = L.r;
        a.R[l] = (const C*)(sizeof(T) == 8 ? (const void*)L.R64 : (const void*)L.R32);
        a.U[l] = (const C*)(sizeof(T) == 8 ? (const void*)L.Ut64 : (const void*)L.Ut32);
        a.S[l] = (const C*)(sizeof(T) == 8 ? (const void*)L.S64 : (const void*)L.S32);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)h.ncta);
    cfg.blockDim = dim3(kHT);
    cfg.dynamicSmemBytes = apply_smem<T>(h);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, hodlr_apply_kernel<T>, a));
}

// Co-resident CTA capacity of the launch (both precisions).
long apply_capacity(const dafmm_hodlr& h)
{
    int dev = 0, sms = 0, p32 = 0, p64 = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t s32 = apply_smem<float>(h), s64 = apply_smem<double>(h);
    CK(cudaFuncSetAttribute(hodlr_apply_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s32));
    CK(cudaFuncSetAttribute(hodlr_apply_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s64));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p32, hodlr_apply_kernel<float>, kHT, s32));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p64, hodlr_apply_kernel<double>, kHT, s64));
    return (long)sms * std::max(0, std::min(p32, p64));
}

// Default width: a power of two, resident at once (two CTAs an SM), at most
// one CTA per leaf, about 256 unknowns per CTA on large problems (at least
// 128 CTAs).  The apply's time falls with the width until the CTAs run out
// (65536 unknowns, rank 15: 194 us at 128 CTAs, 145 us at 256).
int apply_ctas(const dafmm_hodlr& h)
{
    const long want = std::min({h.ncta_cap, h.N / h.leaf, std::max(128L, h.N / 256)});
    long c = 1;
    while (2 * c <= want) c *= 2;
    return (int)c;
}


// ------------------------------------------------------------------------
// Several right-hand sides: x = A~^{-1} b for up to 64 columns stored
// [N][nrhs] (right-hand side fastest).  The steps of the single-column
// launch, as ordinary launches per level (at many columns every step has
// work for the whole GPU, so no grid barrier is needed): the leaf inverses;
// then per level from the leaves up the segment partials of t = W x, the
// node's t and s = S^{-1} t, and x -= Ut s.  Threads take consecutive
// columns, so a vector row is one coalesced access; the factor entries a
// CTA needs and the vector rows it reads are staged in shared memory.  Sums
// run in a fixed order (results do not depend on timing).

constexpr int kBT = 256;     // threads of the several-column kernels
constexpr int kBC = 64;      // columns one CTA covers (nrhs <= 64)
constexpr int kBRows = 64;   // vector rows staged at a time
constexpr int kBQ = 32;      // factor rows staged at a time
constexpr int kBSCols = 16;  // columns per CTA of the s step
constexpr int kBMaxRank = 256;

// x[leaf rows][c] = inv_leaf b[leaf rows][c]; one CTA per leaf.
template <typename T>
__global__ void __launch_bounds__(kBT) hodlr_leaf_many_kernel(int lf, int B, const typename C2<T>::t* __restrict__ inv,
                                                              const double2* __restrict__ b, typename C2<T>::t* __restrict__ x)
{
    using C = typename C2<T>::t;
    using P = Ar<T>;
    using A = typename P::A;
    extern __shared__ __align__(16) unsigned char bsm[];
    C* xs = (C*)bsm;          // rows x B: source rows j0 ..
    C* ms = xs + kBRows * B;  // rows x kBRows: inv[j0 + j][i0 + i] (leaf inverses are column-major)
    const int tid = threadIdx.x, c = tid % kBC, ig = tid / kBC;
    const long l0 = (long)blockIdx.x * lf;
    const C* M = inv + (size_t)blockIdx.x * lf * lf;
    const int rows = min(lf, kBRows);
    for (int i0 = 0; i0 < lf; i0 += rows) {
        A acc[16];
#pragma unroll
        for (int k = 0; k < 16; k++) acc[k] = P::zero();
        for (int j0 = 0; j0 < lf; j0 += rows) {
            __syncthreads();
            for (int e = tid; e < rows * B; e += kBT) xs[e] = P::from64(b[(l0 + j0) * B + e]);
            for (int e = tid; e < rows * rows; e += kBT) {
                const int j = e / rows, i = e - j * rows;
                ms[j * kBRows + i] = M[(size_t)(j0 + j) * lf + i0 + i];
            }
            __syncthreads();
            if (c < B)
                for (int j = 0; j < rows; j++) {
                    const C v = xs[j * B + c];
#pragma unroll
                    for (int k = 0; k < 16; k++)
                        if (ig + 4 * k < rows) P::mac(acc[k], ms[j * kBRows + ig + 4 * k], v);
                }
        }
        if (c < B)
#pragma unroll
            for (int k = 0; k < 16; k++)
                if (ig + 4 * k < rows) x[(l0 + i0 + ig + 4 * k) * B + c] = P::to_c(acc[k]);
    }
}

// part[g][q][c] = sum over the seg rows i of segment g of R[q][i] x[i][c]; one CTA per segment.
template <typename T>
__global__ void __launch_bounds__(kBT) hodlr_wx_many_kernel(long N, int B, int r, long seg, const typename C2<T>::t* __restrict__ R,
                                                            const typename C2<T>::t* __restrict__ x, typename C2<T>::t* __restrict__ part)
{
    using C = typename C2<T>::t;
    using P = Ar<T>;
    using A = typename P::A;
    extern __shared__ __align__(16) unsigned char bsm[];
    C* xs = (C*)bsm;          // rows x B
    C* rs = xs + kBRows * B;  // kBQ x kBRows: R[q0 + q][i0 + i]
    const int tid = threadIdx.x, c = tid % kBC, qg = tid / kBC;
    const long s0 = (long)blockIdx.x * seg;
    const int rows = (int)min(seg, (long)kBRows);
    for (int q0 = 0; q0 < r; q0 += kBQ) {
        const int qn = min(kBQ, r - q0);
        A acc[kBQ / 4];
#pragma unroll
        for (int k = 0; k < kBQ / 4; k++) acc[k] = P::zero();
        for (long i0 = s0; i0 < s0 + seg; i0 += rows) {
            __syncthreads();
            for (int e = tid; e < rows * B; e += kBT) xs[e] = x[i0 * B + e];
            for (int e = tid; e < qn * rows; e += kBT) {
                const int q = e / rows, i = e - q * rows;
                rs[q * kBRows + i] = R[(size_t)(q0 + q) * N + i0 + i];
            }
            __syncthreads();
            if (c < B)
                for (int i = 0; i < rows; i++) {
                    const C v = xs[i * B + c];
#pragma unroll
                    for (int k = 0; k < kBQ / 4; k++)
                        if (qg + 4 * k < qn) P::mac(acc[k], rs[(qg + 4 * k) * kBRows + i], v);
                }
        }
        if (c < B)
#pragma unroll
            for (int k = 0; k < kBQ / 4; k++)
                if (qg + 4 * k < qn) part[((size_t)blockIdx.x * r + q0 + qg + 4 * k) * B + c] = P::to_c(acc[k]);
    }
}

// Node blockIdx.x, columns blockIdx.y * 16 ..: t (rows [0, r) from the partials of
// half 2's segments, rows [r, 2r) from half 1's, summed in segment order), then
// s = S^{-1} t into sout[node][2 r][c].
template <typename T>
__global__ void __launch_bounds__(kBT) hodlr_s_many_kernel(int B, int r, long gper, const typename C2<T>::t* __restrict__ part,
                                                           const typename C2<T>::t* __restrict__ S, typename C2<T>::t* __restrict__ sout)
{
    using C = typename C2<T>::t;
    using P = Ar<T>;
    using A = typename P::A;
    extern __shared__ __align__(16) unsigned char bsm[];
    C* ts = (C*)bsm;  // 2 r x kBSCols
    const int tid = threadIdx.x, cl = tid % kBSCols, ag = tid / kBSCols;
    constexpr int kG = kBT / kBSCols;
    const int c = blockIdx.y * kBSCols + cl;
    const long nd = blockIdx.x;
    const int R2 = 2 * r;
    for (int a = ag; a < R2; a += kG) {
        A acc = P::zero();
        if (c < B) {
            const long g0 = nd * 2 * gper + (a < r ? gper : 0);
            const int q = a < r ? a : a - r;
            for (long g = 0; g < gper; g++) P::add_c(acc, part[((g0 + g) * r + q) * B + c]);
        }
        ts[a * kBSCols + cl] = P::to_c(acc);
    }
    __syncthreads();
    const C* Sn = S + (size_t)nd * 4 * r * r;
    for (int a = ag; a < R2; a += kG) {
        A acc = P::zero();
        for (int bb = 0; bb < R2; bb++) P::mac(acc, Sn[(size_t)a * R2 + bb], ts[bb * kBSCols + cl]);
        if (c < B) sout[((size_t)nd * R2 + a) * B + c] = P::to_c(acc);
    }
}

// x[i][c] -= sum_q Ut[q][i] s[node][hoff + q][c] on the tile of blockIdx.x
// (tile rows, inside one half of one node).
template <typename T>
__global__ void __launch_bounds__(kBT) hodlr_upd_many_kernel(long N, int B, int r, long n, int tile, const typename C2<T>::t* __restrict__ U,
                                                             const typename C2<T>::t* __restrict__ sbuf, typename C2<T>::t* __restrict__ x)
{
    using C = typename C2<T>::t;
    using P = Ar<T>;
    using A = typename P::A;
    extern __shared__ __align__(16) unsigned char bsm[];
    C* ss = (C*)bsm;        // kBQ x B
    C* us = ss + kBQ * B;   // kBQ x kBRows
    const int tid = threadIdx.x, c = tid % kBC, ig = tid / kBC;
    const long i0 = (long)blockIdx.x * tile;
    const long nd = i0 / n;
    const int hoff = (i0 - nd * n) >= n / 2 ? r : 0;
    const C* sn = sbuf + ((size_t)nd * 2 * r + hoff) * B;
    A acc[16];
#pragma unroll
    for (int k = 0; k < 16; k++) acc[k] = P::zero();
    for (int q0 = 0; q0 < r; q0 += kBQ) {
        const int qn = min(kBQ, r - q0);
        __syncthreads();
        for (int e = tid; e < qn * B; e += kBT) ss[e] = sn[(size_t)q0 * B + e];
        for (int e = tid; e < qn * tile; e += kBT) {
            const int q = e / tile, i = e - q * tile;
            us[q * kBRows + i] = U[(size_t)(q0 + q) * N + i0 + i];
        }
        __syncthreads();
        if (c < B)
            for (int q = 0; q < qn; q++) {
                const C sv = ss[q * B + c];
#pragma unroll
                for (int k = 0; k < 16; k++)
                    if (ig + 4 * k < tile) P::mac(acc[k], us[q * kBRows + ig + 4 * k], sv);
            }
    }
    if (c < B)
#pragma unroll
        for (int k = 0; k < 16; k++)
            if (ig + 4 * k < tile) {
                C* xp = x + (i0 + ig + 4 * k) * B + c;
                *xp = P::sub(*xp, acc[k]);
            }
}

template <typename T>
__global__ void hodlr_out_many_kernel(long n, const typename C2<T>::t* __restrict__ x, double2* __restrict__ out)
{
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e < n) out[e] = Ar<T>::to64(x[e]);
}

// Segment length of level l for the several-column partials: the half, capped
// so that a level has at least about 256 segments (one CTA each).
long many_seg(const dafmm_hodlr& h, int l)
{
    const long half = (h.N >> l) / 2;
    return std::min(half, std::max(64L, h.N / 256));
}

template <typename T>
size_t many_smem(int kind, int B)
{
    using C = typename C2<T>::t;
    switch (kind) {
        case 0: return sizeof(C) * (size_t)(kBRows * B + kBRows * kBRows);  // leaf
        case 1: return sizeof(C) * (size_t)(kBRows * B + kBQ * kBRows);     // W x
        case 2: return sizeof(C) * (size_t)(2 * kBMaxRank * kBSCols);       // s
        default: return sizeof(C) * (size_t)(kBQ * B + kBQ * kBRows);       // update
    }
}

void ensure_many(dafmm_hodlr& h, int B)
{
    if (h.bcap >= B) return;
    cudaFree(h.bx);
    cudaFree(h.bpart);
    cudaFree(h.bs);
    h.bx = h.bpart = h.bs = nullptr;
    h.bcap = 0;
    size_t npart = 1, ns = 1;
    for (int l = 0; l < h.H; l++) {
        const int r = h.dlv[l].r;
        npart = std::max(npart, (size_t)(h.N / many_seg(h, l)) * r);
        ns = std::max(ns, (size_t)(1L << l) * 2 * r);
    }
    if (cudaMalloc(&h.bx, sizeof(double2) * (size_t)h.N * B) != cudaSuccess ||
        cudaMalloc(&h.bpart, sizeof(double2) * npart * B) != cudaSuccess || cudaMalloc(&h.bs, sizeof(double2) * ns * B) != cudaSuccess) {
        cudaGetLastError();
        fail(DAFMM_ENOMEM, "device allocation for the several-right-hand-side HODLR buffers failed");
    }
    h.bcap = B;
    {  // the handle's device (attributes are set per device)
        CK(cudaFuncSetAttribute(hodlr_leaf_many_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)many_smem<double>(0, kBC)));
        CK(cudaFuncSetAttribute(hodlr_leaf_many_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)many_smem<float>(0, kBC)));
        CK(cudaFuncSetAttribute(hodlr_wx_many_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)many_smem<double>(1, kBC)));
        CK(cudaFuncSetAttribute(hodlr_wx_many_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)many_smem<float>(1, kBC)));
        CK(cudaFuncSetAttribute(hodlr_s_many_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)many_smem<double>(2, kBC)));
        CK(cudaFuncSetAttribute(hodlr_s_many_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)many_smem<float>(2, kBC)));
        CK(cudaFuncSetAttribute(hodlr_upd_many_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)many_smem<double>(3, kBC)));
        CK(cudaFuncSetAttribute(hodlr_upd_many_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)many_smem<float>(3, kBC)));
    }
}

template <typename T>
void apply_many(dafmm_hodlr& h, int B, const double2* b, double2* xout, cudaStream_t s)
{
    using C = typename C2<T>::t;
    ensure_many(h, B);
    C* x = (C*)h.bx;
    C* part = (C*)h.bpart;
    C* sb = (C*)h.bs;
    const C* inv = (const C*)(sizeof(T) == 8 ? (const void*)h.inv64 : (const void*)h.inv32);
    hodlr_leaf_many_kernel<T><<<(unsigned)(h.N / h.leaf), kBT, many_smem<T>(0, B), s>>>(h.leaf, B, inv, b, x);
    for (int l = h.H - 1; l >= 0; l--) {
        const HodlrDevLevel& L = h.dlv[l];
        const int r = L.r;
        if (r == 0) continue;
        const long n = h.N >> l, half = n / 2, seg = many_seg(h, l);
        const C* R = (const C*)(sizeof(T) == 8 ? (const void*)L.R64 : (const void*)L.R32);
        const C* U = (const C*)(sizeof(T) == 8 ? (const void*)L.Ut64 : (const void*)L.Ut32);
        const C* S = (const C*)(sizeof(T) == 8 ? (const void*)L.S64 : (const void*)L.S32);
        hodlr_wx_many_kernel<T><<<(unsigned)(h.N / seg), kBT, many_smem<T>(1, B), s>>>(h.N, B, r, seg, R, x, part);
        hodlr_s_many_kernel<T><<<dim3((unsigned)(h.N / n), (unsigned)((B + kBSCols - 1) / kBSCols)), kBT, sizeof(C) * 2 * r * kBSCols, s>>>(
            B, r, half / seg, part, S, sb);
        const int tile = (int)std::min<long>(kBRows, half);
        hodlr_upd_many_kernel<T><<<(unsigned)(h.N / tile), kBT, many_smem<T>(3, B), s>>>(h.N, B, r, n, tile, U, sb, x);
    }
    const long ne = h.N * (long)B;
    hodlr_out_many_kernel<T><<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(ne, x, xout);
}

}  // namespace

const dafmm_tree* hodlr_tree(const dafmm_hodlr* h) { return h->tree; }

void hodlr_apply_many(const dafmm_hodlr* h, int nrhs, const double* b, double* x, int precision, cudaStream_t s)
{
    cudaGetLastError();
    if (nrhs < 1 || nrhs > kBC) fail(DAFMM_EBADARG, "hodlr_solve takes 1 to 64 right-hand sides");
    if (h->rmax > kBMaxRank) fail(DAFMM_EBADARG, "several right-hand sides need HODLR ranks of at most 256");
    dafmm_hodlr& hm = const_cast<dafmm_hodlr&>(*h);  // work buffers only
    if (precision == DAFMM_FP64)
        apply_many<double>(hm, nrhs, (const double2*)b, (double2*)x, s);
    else
        apply_many<float>(hm, nrhs, (const double2*)b, (double2*)x, s);
    CK(cudaGetLastError());
}

void hodlr_apply(const dafmm_hodlr* h, const double* b, double* x, int precision, cudaStream_t s)
{
    cudaGetLastError();
    if (precision == DAFMM_FP64)
        apply<double>(*h, (const double2*)b, (double2*)x, s);
    else
        apply<float>(*h, (const double2*)b, (double2*)x, s);
    CK(cudaGetLastError());
}

int hodlr_check(const dafmm_hodlr* h, cudaStream_t s)
{
    CK(cudaStreamSynchronize(s));
    int flag = 0;
    CK(cudaMemcpy(&flag, h->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!flag) return DAFMM_OK;
    // a launch that gave up may have left the barrier armed
    CK(cudaMemset(h->bar, 0, 2 * sizeof(unsigned)));
    CK(cudaMemset(h->err, 0, sizeof(int)));
    return DAFMM_ETIMEOUT;
}

void hodlr_set_stall(const dafmm_hodlr* h, int on) { h->stall = on ? 1 : 0; }

void hodlr_set_width(dafmm_hodlr* h, int ctas)
{
    if (ctas == 0) {
        h->ncta = h->ncta_default;
        return;
    }
    if (ctas < 0 || (ctas & (ctas - 1)) || ctas > h->N / h->leaf || ctas > h->ncta_cap)
        fail(DAFMM_EBADARG, "CTAs must be a power of two, at most one per leaf (" + std::to_string(h->N / h->leaf) +
                                ") and at most the resident capacity (" + std::to_string(h->ncta_cap) + ")");
    h->ncta = ctas;
}

void hodlr_prec(const void* M, const double* v, double* z, int precision, cudaStream_t s)
{
    hodlr_apply((const dafmm_hodlr*)M, v, z, precision, s);
}

void hodlr_prec_many(const void* M, int nrhs, const double* v, double* z, int precision, cudaStream_t s)
{
    hodlr_apply_many((const dafmm_hodlr*)M, nrhs, v, z, precision, s);
}

dafmm_hodlr* hodlr_build(const dafmm_ops* ops, int rank, double tol, int leaf)
{
    auto t0 = std::chrono::steady_clock::now();
    const Tree& t = ops->tree->t;
    const long N = t.N;
    if (leaf < 32 || (leaf & (leaf - 1)) || leaf > 1024) fail(DAFMM_EBADARG, "leaf size must be a power of two in 32..1024");
    if (rank < 0 || (rank == 0 && !(tol > 0 && tol < 1))) fail(DAFMM_EBADARG, "give rank > 0, or rank = 0 and tol in (0, 1)");
    if (rank > 1024) fail(DAFMM_EBADARG, "rank above 1024");
    dafmm_hodlr* h = new dafmm_hodlr();
    try {
        h->tree = ops->tree;
        h->N = N;
        h->leaf = (int)std::min<long>(leaf, N);
        int H = 0;
        while ((N >> H) > h->leaf) H++;
        if (H > kHodlrMaxLevels) fail(DAFMM_EBADARG, "too many HODLR levels; use a larger leaf size");
        h->H = H;
        // contrast on the host: A_ij = delta_ij + kappa^2 q_i K_ij
        std::vector<double> q(N);
        CK(cudaMemcpy(q.data(), ops->dev.q, sizeof(double) * N, cudaMemcpyDeviceToHost));
        const double k2 = t.prm.kappa * t.prm.kappa;
        const EntryTable& K = ops->table;
        auto A = [&](long i, long j) { return (i == j ? cd(1.0) : cd(0.0)) + k2 * q[i] * K(i, j); };
        const int lf = h->leaf;
        const long nleaf = N / lf;
        h->leafA.assign((size_t)nleaf * lf * lf, cd(0));
        h->leafInv.resize(h->leafA.size());
        std::vector<int> bad(nleaf, 0);
#pragma omp parallel for schedule(dynamic, 4)
        for (long b = 0; b < nleaf; b++) {
            std::vector<cd> a((size_t)lf * lf);
            for (int i = 0; i < lf; i++)
                for (int j = 0; j < lf; j++) a[(size_t)i * lf + j] = A(b * lf + i, b * lf + j);
            std::copy(a.begin(), a.end(), h->leafA.begin() + (size_t)b * lf * lf);
            if (!invert(a, lf)) bad[b] = 1;
            std::copy(a.begin(), a.end(), h->leafInv.begin() + (size_t)b * lf * lf);
        }
        for (int v : bad)
            if (v) fail(DAFMM_EBREAKDOWN, "singular HODLR leaf block");
        h->lv.assign(H, HodlrLevelHost());
        for (int l = H - 1; l >= 0; l--) {
            const long n = N >> l, half = n / 2, nodes = N / n;
            HodlrLevelHost& L = h->lv[l];
            // compress the off-diagonal blocks of every node
            std::vector<std::vector<std::vector<cd>>> U12(nodes), V12(nodes), U21(nodes), V21(nodes);
#pragma omp parallel for schedule(dynamic, 1)
            for (long k = 0; k < nodes; k++) {
                std::vector<long> I1(half), I2(half);
                for (long i = 0; i < half; i++) {
                    I1[i] = k * n + i;
                    I2[i] = k * n + half + i;
                }
                AcaPivots pv;
                aca_run(A, I1, I2, rank > 0 ? 0.0 : tol, rank, pv, &U12[k], &V12[k]);
                aca_run(A, I2, I1, rank > 0 ? 0.0 : tol, rank, pv, &U21[k], &V21[k]);
            }
            int r = 0;
            for (long k = 0; k < nodes; k++) r = std::max(r, (int)std::max(U12[k].size(), U21[k].size()));
            L.r = r;
            L.R.assign((size_t)r * N, cd(0));
            L.U.assign((size_t)N * r, cd(0));
            L.Ut.assign((size_t)N * r, cd(0));
            L.Sinv.assign((size_t)nodes * 4 * r * r, cd(0));
            std::vector<int> sing(nodes, 0);
#pragma omp parallel for schedule(dynamic, 1)
            for (long k = 0; k < nodes; k++) {
                const long i0 = k * n;
                for (size_t q = 0; q < V21[k].size(); q++)
                    for (long i = 0; i < half; i++) L.R[q * N + i0 + i] = V21[k][q][i];
                for (size_t q = 0; q < V12[k].size(); q++)
                    for (long i = 0; i < half; i++) L.R[q * N + i0 + half + i] = V12[k][q][i];
                // Ut = D^{-1} diag(U12, U21): apply the children's inverses
                std::vector<std::vector<cd>> c1(r, std::vector<cd>(half, cd(0))), c2(r, std::vector<cd>(half, cd(0)));
                for (size_t q = 0; q < U12[k].size(); q++) c1[q] = U12[k][q];
                for (size_t q = 0; q < U21[k].size(); q++) c2[q] = U21[k][q];
                for (int q = 0; q < r; q++)
                    for (long i = 0; i < half; i++) {
                        L.U[(size_t)(i0 + i) * r + q] = c1[q][i];
                        L.U[(size_t)(i0 + half + i) * r + q] = c2[q][i];
                    }
                host_solve(*h, l + 1, 2 * k, c1);
                host_solve(*h, l + 1, 2 * k + 1, c2);
                for (int q = 0; q < r; q++)
                    for (long i = 0; i < half; i++) {
                        L.Ut[(size_t)(i0 + i) * r + q] = c1[q][i];
                        L.Ut[(size_t)(i0 + half + i) * r + q] = c2[q][i];
                    }
                // S = I + [[0, V12 Ut2], [V21 Ut1, 0]]
                std::vector<cd> S((size_t)4 * r * r, cd(0));
                for (int a = 0; a < 2 * r; a++) S[(size_t)a * 2 * r + a] = 1.0;
                for (int a = 0; a < r; a++)
                    for (int b = 0; b < r; b++) {
                        cd v12 = 0, v21 = 0;
                        for (long i = 0; i < half; i++) {
                            v12 += L.R[(size_t)a * N + i0 + half + i] * c2[b][i];
                            v21 += L.R[(size_t)a * N + i0 + i] * c1[b][i];
                        }
                        S[(size_t)a * 2 * r + r + b] += v12;
                        S[(size_t)(r + a) * 2 * r + b] += v21;
                    }
                if (!invert(S, 2 * r)) sing[k] = 1;
                std::copy(S.begin(), S.end(), L.Sinv.begin() + (size_t)k * 4 * r * r);
            }
            for (int v : sing)
                if (v) fail(DAFMM_EBREAKDOWN, "singular Woodbury system in the HODLR factorisation");
        }
        // upload: leaf inverses column-major, level factors, work buffers
        std::vector<cd> invc(h->leafInv.size());
        for (long b = 0; b < nleaf; b++)
            for (int i = 0; i < lf; i++)
                for (int j = 0; j < lf; j++)
                    invc[(size_t)b * lf * lf + (size_t)j * lf + i] = h->leafInv[(size_t)b * lf * lf + (size_t)i * lf + j];
        up(to_pairs(invc), &h->inv64);
        up(to32(invc), &h->inv32);
        h->dlv.assign(H, HodlrDevLevel());
        for (int l = 0; l < H; l++) {
            HodlrDevLevel& D = h->dlv[l];
            const HodlrLevelHost& L = h->lv[l];
            D.r = L.r;
            h->rmax = std::max(h->rmax, L.r);
            up(to_pairs(L.R), &D.R64);
            up(to32(L.R), &D.R32);
            // Ut as r x N, so that the update reads it along the unknowns
            std::vector<cd> utt((size_t)L.r * N);
            for (long i = 0; i < N; i++)
                for (int q = 0; q < L.r; q++) utt[(size_t)q * N + i] = L.Ut[(size_t)i * L.r + q];
            up(to_pairs(utt), &D.Ut64);
            up(to32(utt), &D.Ut32);
            up(to_pairs(L.Sinv), &D.S64);
            up(to32(L.Sinv), &D.S32);
        }
        const long nl = std::max<long>(N / h->leaf, 1);
        h->sbuf_half = 2L * std::max(1, h->rmax) * nl;
        if (cudaMalloc(&h->t_part, sizeof(double2) * std::max(1, h->rmax) * nl) != cudaSuccess ||
            cudaMalloc(&h->s_buf, sizeof(double2) * 2 * h->sbuf_half) != cudaSuccess ||
            cudaMalloc(&h->xw, sizeof(float2) * N) != cudaSuccess ||
            cudaMalloc(&h->bar, 2 * sizeof(unsigned)) != cudaSuccess || cudaMalloc(&h->err, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            fail(DAFMM_ENOMEM, "device allocation for the HODLR work buffers failed");
        }
        CK(cudaMemset(h->bar, 0, 2 * sizeof(unsigned)));
        CK(cudaMemset(h->err, 0, sizeof(int)));
        h->ncta_cap = apply_capacity(*h);
        if (h->ncta_cap < 1) fail(DAFMM_EBADARG, "the HODLR apply kernel does not fit an SM (rank too large)");
        h->ncta = h->ncta_default = apply_ctas(*h);
    } catch (...) {
        hodlr_free(h);
        throw;
    }
    h->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return h;
}

void hodlr_free(dafmm_hodlr* h)
{
    if (!h) return;
    cudaFree(h->inv64);
    cudaFree(h->inv32);
    for (auto& D : h->dlv) {
        cudaFree(D.R64);
        cudaFree(D.R32);
        cudaFree(D.Ut64);
        cudaFree(D.Ut32);
        cudaFree(D.S64);
        cudaFree(D.S32);
    }
    cudaFree(h->t_part);
    cudaFree(h->s_buf);
    cudaFree(h->xw);
    cudaFree(h->bar);
    cudaFree(h->err);
    cudaFree(h->bx);
    cudaFree(h->bpart);
    cudaFree(h->bs);
    delete h;
}

void hodlr_shape(const dafmm_hodlr* h, long* N, int* levels, int* leaf, int* rank_max, double* seconds)
{
    *N = h->N;
    *levels = h->H;
    *leaf = h->leaf;
    *rank_max = h->rmax;
    *seconds = h->seconds;
}

// Dense A~ assembled from the factors (row-major, N x N): leaf blocks on the
// diagonal, U12 V12 / U21 V21 off the diagonal at every level.
void hodlr_dense(const dafmm_hodlr* h, cd* out)
{
    const long N = h->N;
    std::fill(out, out + (size_t)N * N, cd(0));
    const int lf = h->leaf;
    for (long b = 0; b < N / lf; b++)
        for (int i = 0; i < lf; i++)
            for (int j = 0; j < lf; j++) out[(size_t)(b * lf + i) * N + b * lf + j] = h->leafA[(size_t)b * lf * lf + (size_t)i * lf + j];
    for (int l = 0; l < h->H; l++) {
        const HodlrLevelHost& L = h->lv[l];
        const long n = N >> l, half = n / 2;
        for (long k = 0; k < N / n; k++) {
            const long i0 = k * n;
#pragma omp parallel for schedule(static)
            for (long i = 0; i < half; i++)
                for (long j = 0; j < half; j++) {
                    cd a12 = 0, a21 = 0;
                    for (int q = 0; q < L.r; q++) {
                        a12 += L.U[(size_t)(i0 + i) * L.r + q] * L.R[(size_t)q * N + i0 + half + j];
                        a21 += L.U[(size_t)(i0 + half + i) * L.r + q] * L.R[(size_t)q * N + i0 + j];
                    }
                    out[(size_t)(i0 + i) * N + i0 + half + j] = a12;
                    out[(size_t)(i0 + half + i) * N + i0 + j] = a21;
                }
        }
    }
}

}  // namespace dafmm
