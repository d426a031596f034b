// GMRES for A psi = f (Eq. 12a) on the device, with optional right
// preconditioning by the HODLR approximation (the Hybrid solver of Section
// 6, Eq. hybrid) and FP64 iterative refinement around mixed-precision inner
// cycles.
//
// Outer step k: r = f - A x with the FP64 DAFMM; stop when |r|/|f| <= tol
// (the stopping rule of Section 6, relative residual of the unpreconditioned
// system).  Otherwise one flexible GMRES(m) cycle solves A d = r with
// operators in the requested precision, and x += d.  With FP64 inner
// operators this is restarted GMRES with the true residual checked at every
// restart; with mixed inner operators it is iterative refinement whose
// correction equations are solved to a relative inner tolerance.
//
// Arnoldi is classical Gram-Schmidt applied twice; the Hessenberg matrix, the
// Givens rotations, the preconditioned basis and x stay in FP64 on the
// device, the Arnoldi basis is complex128 in FP64 cycles and complex64 in the
// inner cycles of mixed precision (whose target is a relative 1e-5).  One
// Arnoldi step is three reduction kernels (the last block of each sums the
// per-block partials in block order, so results do not depend on timing) and
// a scaling; the host reads one residual estimate (8 bytes) per step to
// decide when to stop.  While it waits for step j it may already have queued
// step j + 1 when the estimates so far predict that step j misses the target
// by far (geometric extrapolation); a step queued that way and not needed
// writes only columns the final update does not read.  A zero initial guess
// takes r = f without an application.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

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

constexpr int kAT = 256;  // threads per block of the reduction kernels
constexpr int kCR = 64;   // rows per block: the block stages V[rows, 0..nk) in shared memory
constexpr int kMaxM = 128;
constexpr int kThreads = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// True in the last block of the grid to get here (its partials and everyone
// else's are visible to it); that block re-arms the ticket.
__device__ bool last_block(unsigned* ticket)
{
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        if (last) *ticket = 0;
        s_last = last;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// Basis vectors: complex128 (FP64 cycles) or complex64 (the inner cycles of
// mixed precision, where the correction equation is solved to ~1e-5).
template <typename T>
struct CT;
template <>
struct CT<double> {
    using t = double2;
};
template <>
struct CT<float> {
    using t = float2;
};

template <typename C>
__device__ __forceinline__ C cmul_t(C a, C b)
{
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

template <typename C>
__device__ __forceinline__ C cconjmul_t(C a, C b)  // conj(a) * b
{
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.x * b.y - a.y * b.x;
    return r;
}

template <typename T>
__device__ __forceinline__ typename CT<T>::t from64(double2 v)
{
    typename CT<T>::t r;
    r.x = (T)v.x;
    r.y = (T)v.y;
    return r;
}

// Vs[k][r] = V[r0 + r, k] for r < rows, k < nk, by asynchronous copies (all in
// flight at once), then wait.
template <typename T>
__device__ __forceinline__ void stage_tile(const typename CT<T>::t* __restrict__ V, long N, int nk, long r0, int rows, typename CT<T>::t* Vs)
{
    for (int e = threadIdx.x; e < nk * kCR; e += blockDim.x) {
        const int k = e / kCR, r = e - k * kCR;
        if (r < rows) {
            const unsigned dst = (unsigned)__cvta_generic_to_shared(Vs + e);
            if constexpr (sizeof(T) == 8)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(V + (size_t)k * N + r0 + r) : "memory");
            else
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(V + (size_t)k * N + r0 + r) : "memory");
        }
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    __syncthreads();
}

// ws[r] = w[r0 + r] - sum_k Vs[k][r] h[k] (hs == nullptr: no update), four
// threads per row splitting k; rows past the end are zero.  With w64 the row
// is read from that complex128 vector instead (and rounded to T).  Writes the
// rows back to w when they changed (hs or w64 given).
template <typename T>
__device__ __forceinline__ void tile_update(const typename CT<T>::t* Vs, int nk, const typename CT<T>::t* hs, typename CT<T>::t* __restrict__ w,
                                            const double2* __restrict__ w64, long r0, int rows, typename CT<T>::t* ws)
{
    using C = typename CT<T>::t;
    const int r = threadIdx.x >> 2, part = threadIdx.x & 3;  // kAT = 4 kCR
    C a;
    a.x = 0;
    a.y = 0;
    if (hs)
        for (int k = part; k < nk; k += 4) {
            const C p = cmul_t(Vs[k * kCR + r], hs[k]);
            a.x += p.x;
            a.y += p.y;
        }
    for (int o = 1; o < 4; o <<= 1) {
        a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
        a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
    }
    if (part == 0) {
        C v;
        v.x = 0;
        v.y = 0;
        if (r < rows) {
            v = w64 ? from64<T>(w64[r0 + r]) : w[r0 + r];
            v.x -= a.x;
            v.y -= a.y;
            if (hs || w64) w[r0 + r] = v;
        }
        ws[r] = v;
    }
    __syncthreads();
}

// Sum over blocks of part[k][*] for k < nk into out (last block, warp per k).
__device__ __forceinline__ void reduce_blocks(const double2* part, int nk, int nrb, double2* out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kW = kAT / 32;
    for (int k0 = warp; k0 < nk; k0 += 2 * kW) {
        double2 t[2] = {make_double2(0, 0), make_double2(0, 0)};
#pragma unroll 8
        for (int rb = lane; rb < nrb; rb += 32)
#pragma unroll
            for (int u = 0; u < 2; u++)
                if (k0 + u * kW < nk) {
                    const double2 p = __ldcg(&part[(size_t)(k0 + u * kW) * nrb + rb]);
                    t[u].x += p.x;
                    t[u].y += p.y;
                }
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int u = 0; u < 2; u++) {
                t[u].x += __shfl_xor_sync(0xffffffffu, t[u].x, o);
                t[u].y += __shfl_xor_sync(0xffffffffu, t[u].y, o);
            }
        if (lane < 2 && k0 + lane * kW < nk) out[k0 + lane * kW] = lane ? t[1] : t[0];
    }
}

// out[0..nk) = V[:, 0..nk)^H w, after w -= V h_in when h_in is given (w read
// from w64 when that is given).  Products and per-block sums in T, block
// partials summed in FP64.  Dynamic shared memory: nk kCR entries of T's
// complex type.  part: nk x gridDim.x partials.
template <typename T>
__global__ void __launch_bounds__(kAT) cgs_kernel(long N, const typename CT<T>::t* __restrict__ V, int nk, const double2* __restrict__ h_in,
                                                  typename CT<T>::t* __restrict__ w, const double2* __restrict__ w64,
                                                  double2* __restrict__ part, unsigned* ticket, double2* __restrict__ out)
{
    using C = typename CT<T>::t;
    extern __shared__ __align__(16) unsigned char cgs_smem[];
    C* Vs = (C*)cgs_smem;
    __shared__ C hs[kMaxM + 1];
    __shared__ C ws[kCR];
    const long r0 = (long)blockIdx.x * kCR;
    const int rows = (int)min((long)kCR, N - r0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nrb = gridDim.x;
    if (h_in)
        for (int k = threadIdx.x; k < nk; k += blockDim.x) hs[k] = from64<T>(h_in[k]);
    stage_tile<T>(V, N, nk, r0, rows, Vs);
    tile_update<T>(Vs, nk, h_in ? hs : nullptr, w, w64, r0, rows, ws);
    // column k by warp k % 8, lanes over the rows
    for (int k = warp; k < nk; k += kAT / 32) {
        C p;
        p.x = 0;
        p.y = 0;
        for (int r = lane; r < kCR; r += 32) {
            const C q = cconjmul_t(Vs[k * kCR + r], ws[r]);
            p.x += r < rows ? q.x : (T)0;
            p.y += r < rows ? q.y : (T)0;
        }
        for (int o = 16; o > 0; o >>= 1) {
            p.x += __shfl_xor_sync(0xffffffffu, p.x, o);
            p.y += __shfl_xor_sync(0xffffffffu, p.y, o);
        }
        if (lane == 0) part[(size_t)k * nrb + blockIdx.x] = make_double2(p.x, p.y);
    }
    if (!last_block(ticket)) return;
    reduce_blocks(part, nk, nrb, out);
}

// Givens bookkeeping for column j by one warp: h[0..j] = h1 + h2, h[j+1] =
// |w| and the previous rotations are staged in shared memory by the warp;
// lane 0 applies the rotations (they chain), forms the new one, updates g
// and publishes |g[j+1]| (the residual norm of the least-squares problem);
// the warp writes the column back.  H is (m+1) x m column-major.
__device__ void givens_step(int j, int m, const double2* h1, const double2* h2, double wn2, double2* H, double2* cs, double2* sn, double2* g,
                            double* res)
{
    __shared__ double2 col[kMaxM + 1], ss[kMaxM];
    __shared__ double cc[kMaxM];
    const int lane = threadIdx.x & 31;
    for (int k = lane; k <= j; k += 32) col[k] = make_double2(__ldcg(&h1[k]).x + __ldcg(&h2[k]).x, __ldcg(&h1[k]).y + __ldcg(&h2[k]).y);
    for (int k = lane; k < j; k += 32) {
        cc[k] = cs[k].x;
        ss[k] = sn[k];
    }
    __syncwarp();
    if (lane == 0) {
        col[j + 1] = make_double2(sqrt(wn2), 0.0);
        // previous rotations: [c s; -conj(s) c] with real c
        for (int k = 0; k < j; k++) {
            const double c = cc[k];
            const double2 s = ss[k];
            const double2 a = col[k], b = col[k + 1];
            const double2 sb = cmul(s, b);
            const double2 csa = make_double2(s.x * a.x + s.y * a.y, s.x * a.y - s.y * a.x);  // conj(s) a
            col[k] = make_double2(c * a.x + sb.x, c * a.y + sb.y);
            col[k + 1] = make_double2(-csa.x + c * b.x, -csa.y + c * b.y);
        }
        // new rotation zeroing col[j+1]
        const double2 a = col[j], b = col[j + 1];
        const double na = hypot(a.x, a.y), nb = hypot(b.x, b.y);
        double c;
        double2 s;
        if (nb == 0.0) {
            c = 1.0;
            s = make_double2(0, 0);
        } else if (na == 0.0) {
            c = 0.0;
            s = make_double2(b.x / nb, -b.y / nb);  // conj(b)/|b|
        } else {
            const double t = hypot(na, nb);
            c = na / t;
            const double2 ua = make_double2(a.x / na, a.y / na);  // a/|a|
            // s = (a/|a|) conj(b) / t
            s = make_double2((ua.x * b.x + ua.y * b.y) / t, (ua.y * b.x - ua.x * b.y) / t);
        }
        cs[j] = make_double2(c, 0.0);
        sn[j] = s;
        const double2 sb = cmul(s, b);
        col[j] = make_double2(c * a.x + sb.x, c * a.y + sb.y);
        col[j + 1] = make_double2(0.0, 0.0);
        const double2 gj = g[j];
        const double2 csg = make_double2(s.x * gj.x + s.y * gj.y, s.x * gj.y - s.y * gj.x);  // conj(s) g_j
        g[j] = make_double2(c * gj.x, c * gj.y);
        g[j + 1] = make_double2(-csg.x, -csg.y);
        *res = hypot(g[j + 1].x, g[j + 1].y);
    }
    __syncwarp();
    double2* hc = H + (size_t)j * (m + 1);
    for (int k = lane; k <= j + 1; k += 32) hc[k] = col[k];
}

struct GivensArgs {
    int j, m;
    const double2 *h1, *h2;
    double2 *H, *cs, *sn, *g;
    double* res;
};

// w -= V h_in (h_in may be null), then |w|^2 -> *wn2 (real part); with
// gv.H, the last block also takes the Givens step of column gv.j.
// Dynamic shared memory: nk kCR entries.  part: gridDim.x partials.
template <typename T>
__global__ void __launch_bounds__(kAT) cgs_norm_kernel(long N, const typename CT<T>::t* __restrict__ V, int nk, const double2* __restrict__ h_in,
                                                       typename CT<T>::t* __restrict__ w, double2* __restrict__ part, unsigned* ticket,
                                                       double2* __restrict__ wn2, GivensArgs gv)
{
    using C = typename CT<T>::t;
    extern __shared__ __align__(16) unsigned char cgs_smem[];
    C* Vs = (C*)cgs_smem;
    __shared__ C hs[kMaxM + 1];
    __shared__ C ws[kCR];
    __shared__ double red[kAT / 32];
    const long r0 = (long)blockIdx.x * kCR;
    const int rows = (int)min((long)kCR, N - r0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nrb = gridDim.x;
    if (h_in)
        for (int k = threadIdx.x; k < nk; k += blockDim.x) hs[k] = from64<T>(h_in[k]);
    if (h_in) stage_tile<T>(V, N, nk, r0, rows, Vs);
    tile_update<T>(Vs, h_in ? nk : 0, h_in ? hs : nullptr, w, nullptr, r0, rows, ws);
    if (warp == 0) {
        double s2 = 0;
        for (int r = lane; r < kCR; r += 32) s2 += (double)ws[r].x * ws[r].x + (double)ws[r].y * ws[r].y;
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0) red[0] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(red[0], 0.0);
    if (!last_block(ticket)) return;
    if (warp == 0) {
        double t = 0;
#pragma unroll 8
        for (int rb = lane; rb < nrb; rb += 32) t += __ldcg(&part[rb]).x;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) *wn2 = make_double2(t, 0.0);
        if (gv.H) givens_step(gv.j, gv.m, gv.h1, gv.h2, t, gv.H, gv.cs, gv.sn, gv.g, gv.res);
    }
}

// x[i] += sum_{k<nk} Z[i, k] y[k]  (Z complex128 or complex64)
template <typename C>
__global__ void __launch_bounds__(kThreads) add_zy_kernel(long N, const C* __restrict__ Z, long ldz, int nk, const double2* __restrict__ y,
                                                          double2* __restrict__ x)
{
    __shared__ double2 ys[kMaxM];
    for (int k = threadIdx.x; k < nk; k += blockDim.x) ys[k] = y[k];
    __syncthreads();
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double2 a = x[i];
#pragma unroll 8
    for (int k = 0; k < nk; k++) {
        const C z = Z[(size_t)k * ldz + i];
        const double2 p = cmul(make_double2((double)z.x, (double)z.y), ys[k]);
        a.x += p.x;
        a.y += p.y;
    }
    x[i] = a;
}

// out = a / sqrt(re(*nrm2)) (0 when the norm is 0), a read from a (T) or a64
// (complex128); written to out (T) and, when given, out64 (complex128).
template <typename T>
__global__ void scale_inv_norm_kernel(long N, const typename CT<T>::t* __restrict__ a, const double2* __restrict__ a64,
                                      const double2* __restrict__ nrm2, typename CT<T>::t* __restrict__ out, double2* __restrict__ out64)
{
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double n = sqrt(nrm2->x);
    const double s = n > 0 ? 1.0 / n : 0.0;
    const double2 v = a64 ? a64[i] : make_double2((double)a[i].x, (double)a[i].y);
    const double2 o = make_double2(v.x * s, v.y * s);
    out[i] = from64<T>(o);
    if (out64) out64[i] = o;
}

__global__ void sub_kernel(long N, const double2* __restrict__ a, const double2* __restrict__ b, double2* __restrict__ out)
{
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    out[i] = make_double2(a[i].x - b[i].x, a[i].y - b[i].y);
}

// Back substitution H[0:n,0:n] y = g[0:n], one block of kMaxM threads:
// thread t keeps g[t]; for i from n-1 down, y[i] = g[i] / H[i][i], then every
// t < i subtracts H[t][i] y[i] (column i of H is contiguous).
__global__ void __launch_bounds__(kMaxM) backsolve_kernel(int n, int m, const double2* __restrict__ H, const double2* __restrict__ g,
                                                          double2* __restrict__ y)
{
    __shared__ double2 yi;
    const int t = threadIdx.x;
    double2 gt = t < n ? g[t] : make_double2(0, 0);
    for (int i = n - 1; i >= 0; i--) {
        if (t == i) {
            const double2 d = H[(size_t)i * (m + 1) + i];
            const double dd = d.x * d.x + d.y * d.y;
            const double2 v = dd > 0 ? make_double2((gt.x * d.x + gt.y * d.y) / dd, (gt.y * d.x - gt.x * d.y) / dd) : make_double2(0, 0);
            y[i] = v;
            yi = v;
        }
        __syncthreads();
        if (t < i) {
            const double2 p = cmul(H[(size_t)i * (m + 1) + t], yi);
            gt.x -= p.x;
            gt.y -= p.y;
        }
        __syncthreads();
    }
}

// g = [|r|, 0, ..., 0]
__global__ void init_g_kernel(int m, const double2* __restrict__ rn2, double2* __restrict__ g)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= m) g[k] = k == 0 ? make_double2(sqrt(rn2->x), 0.0) : make_double2(0, 0);
}

unsigned blocks(long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// ------------------------------------------------------------------------
// Several right-hand sides: nrhs independent GMRES processes in lockstep.
// One Arnoldi step applies the preconditioner and the operator to all the
// current basis vectors at once (one batched application each), then every
// column is orthogonalised against its own basis (classical Gram-Schmidt
// twice) by kernels over [N][nrhs] blocks whose threads take consecutive
// columns, and takes its own Givens step.  A column ends its cycle when its
// own estimate reaches its inner tolerance (later steps of that column are
// not used) and leaves the solve when its own FP64 true residual reaches
// tol.  Sums run in a fixed order (results do not depend on timing).

constexpr int kMT = 256;     // threads of the several-column kernels
constexpr int kMB = 64;      // columns at most
constexpr int kMRows = 256;  // rows per CTA of the reductions
constexpr int kMK = 8;       // basis vectors per CTA of the dot products

// w[e] = (w64 ? w64[e] : w[e]) - sum_{k < nk} V_k[e] h[k][c], c = e mod B,
// for the N B entries e of [N][B] vectors (V_k at V + k N B).
template <typename T>
__global__ void many_update_kernel(long NB, int B, const typename CT<T>::t* __restrict__ V, int nk, const double2* __restrict__ h,
                                   typename CT<T>::t* __restrict__ w, const double2* __restrict__ w64)
{
    using C = typename CT<T>::t;
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= NB) return;
    const int c = (int)(e % B);
    C a = w64 ? from64<T>(w64[e]) : w[e];
#pragma unroll 4
    for (int k = 0; k < nk; k++) {
        const C p = cmul_t(V[(size_t)k * NB + e], from64<T>(__ldg(&h[(size_t)k * B + c])));
        a.x -= p.x;
        a.y -= p.y;
    }
    w[e] = a;
}

// part[k][rb][c] = sum over the rows n of block rb of conj(V_k[n][c]) w[n][c],
// for k in [kMK blockIdx.y, + kMK) below nk.  Products and sums in T; the
// four row groups of a block are added in FP64.
template <typename T>
__global__ void __launch_bounds__(kMT) many_dots_kernel(long N, int B, const typename CT<T>::t* __restrict__ V, int nk,
                                                        const typename CT<T>::t* __restrict__ w, double2* __restrict__ part)
{
    using C = typename CT<T>::t;
    __shared__ double2 red[4][kMK][kMB];
    const int tid = threadIdx.x, c = tid % kMB, rg = tid / kMB;
    const long r0 = (long)blockIdx.x * kMRows, r1 = min(N, r0 + kMRows);
    const int k0 = blockIdx.y * kMK, kn = min(kMK, nk - k0);
    const long NB = N * B;
    C acc[kMK];
#pragma unroll
    for (int u = 0; u < kMK; u++) acc[u].x = acc[u].y = 0;
    if (c < B)
        for (long n = r0 + rg; n < r1; n += 4) {
            const C wv = w[n * B + c];
#pragma unroll
            for (int u = 0; u < kMK; u++)
                if (u < kn) {
                    const C p = cconjmul_t(V[(size_t)(k0 + u) * NB + n * B + c], wv);
                    acc[u].x += p.x;
                    acc[u].y += p.y;
                }
        }
#pragma unroll
    for (int u = 0; u < kMK; u++) red[rg][u][c] = make_double2((double)acc[u].x, (double)acc[u].y);
    __syncthreads();
    for (int e = tid; e < kMK * kMB; e += kMT) {
        const int u = e / kMB, cc = e - u * kMB;
        if (u < kn && cc < B) {
            double2 s = red[0][u][cc];
            for (int g = 1; g < 4; g++) {
                s.x += red[g][u][cc].x;
                s.y += red[g][u][cc].y;
            }
            part[((size_t)(k0 + u) * gridDim.x + blockIdx.x) * B + cc] = s;
        }
    }
}

// out[k][c] = sum over rb of part[k][rb][c] (block k; a fixed order).
__global__ void __launch_bounds__(kMT) many_reduce_kernel(int nrb, int B, const double2* __restrict__ part, double2* __restrict__ out)
{
    __shared__ double2 red[4][kMB];
    const int tid = threadIdx.x, c = tid % kMB, g = tid / kMB, k = blockIdx.x;
    double2 a = make_double2(0, 0);
    if (c < B)
        for (int rb = g; rb < nrb; rb += 4) {
            const double2 p = part[((size_t)k * nrb + rb) * B + c];
            a.x += p.x;
            a.y += p.y;
        }
    red[g][c] = a;
    __syncthreads();
    if (g == 0 && c < B)
        out[(size_t)k * B + c] =
            make_double2(red[0][c].x + red[1][c].x + red[2][c].x + red[3][c].x, red[0][c].y + red[1][c].y + red[2][c].y + red[3][c].y);
}

// Givens bookkeeping of step j, one thread per column c: column j of c's
// Hessenberg matrix is h1 + h2 with |w| below it; the previous rotations,
// then a new one zeroing the subdiagonal; g updated, res[c] = |g[j+1]|.
// H: per column (m+1) x m column-major; cs, sn: per column m; g: m + 1.
__global__ void many_givens_kernel(int j, int m, int B, const double2* __restrict__ h1, const double2* __restrict__ h2,
                                   const double2* __restrict__ wn2, double2* __restrict__ H, double2* __restrict__ cs, double2* __restrict__ sn,
                                   double2* __restrict__ g, double* __restrict__ res)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= B) return;
    double2* col = H + ((size_t)c * m + j) * (m + 1);
    double2* csc = cs + (size_t)c * m;
    double2* snc = sn + (size_t)c * m;
    double2* gc = g + (size_t)c * (m + 1);
    for (int k = 0; k <= j; k++) col[k] = make_double2(h1[(size_t)k * B + c].x + h2[(size_t)k * B + c].x, h1[(size_t)k * B + c].y + h2[(size_t)k * B + c].y);
    col[j + 1] = make_double2(sqrt(fmax(wn2[c].x, 0.0)), 0.0);
    for (int k = 0; k < j; k++) {
        const double cc = csc[k].x;
        const double2 s = snc[k];
        const double2 a = col[k], b = col[k + 1];
        const double2 sb = cmul(s, b);
        const double2 csa = make_double2(s.x * a.x + s.y * a.y, s.x * a.y - s.y * a.x);  // conj(s) a
        col[k] = make_double2(cc * a.x + sb.x, cc * a.y + sb.y);
        col[k + 1] = make_double2(-csa.x + cc * b.x, -csa.y + cc * b.y);
    }
    const double2 a = col[j], b = col[j + 1];
    const double na = hypot(a.x, a.y), nb = hypot(b.x, b.y);
    double cc;
    double2 s;
    if (nb == 0.0) {
        cc = 1.0;
        s = make_double2(0, 0);
    } else if (na == 0.0) {
        cc = 0.0;
        s = make_double2(b.x / nb, -b.y / nb);
    } else {
        const double t = hypot(na, nb);
        cc = na / t;
        const double2 ua = make_double2(a.x / na, a.y / na);
        s = make_double2((ua.x * b.x + ua.y * b.y) / t, (ua.y * b.x - ua.x * b.y) / t);
    }
    csc[j] = make_double2(cc, 0.0);
    snc[j] = s;
    const double2 sb = cmul(s, b);
    col[j] = make_double2(cc * a.x + sb.x, cc * a.y + sb.y);
    col[j + 1] = make_double2(0.0, 0.0);
    const double2 gj = gc[j];
    const double2 csg = make_double2(s.x * gj.x + s.y * gj.y, s.x * gj.y - s.y * gj.x);
    gc[j] = make_double2(cc * gj.x, cc * gj.y);
    gc[j + 1] = make_double2(-csg.x, -csg.y);
    res[c] = hypot(gc[j + 1].x, gc[j + 1].y);
}

// out[e] = a[e] / |column c| (0 for a zero norm or an inactive column), a
// read from a (T) or a64 (complex128); written to out (T) and, when given,
// out64 (complex128).
template <typename T>
__global__ void many_scale_kernel(long NB, int B, const typename CT<T>::t* __restrict__ a, const double2* __restrict__ a64,
                                  const double2* __restrict__ nrm2, const int* __restrict__ active, typename CT<T>::t* __restrict__ out,
                                  double2* __restrict__ out64)
{
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= NB) return;
    const int c = (int)(e % B);
    const double n = sqrt(fmax(nrm2[c].x, 0.0));
    const double sc = (n > 0 && active[c]) ? 1.0 / n : 0.0;
    const double2 v = a64 ? a64[e] : make_double2((double)a[e].x, (double)a[e].y);
    const double2 o = make_double2(v.x * sc, v.y * sc);
    out[e] = from64<T>(o);
    if (out64) out64[e] = o;
}

// g[c] = [|r0_c|, 0, ..., 0] for active columns, zero otherwise.
__global__ void many_init_g_kernel(int m, int B, const double2* __restrict__ rn2, const int* __restrict__ active, double2* __restrict__ g)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= B * (m + 1)) return;
    const int c = e / (m + 1), k = e - c * (m + 1);
    g[e] = (k == 0 && active[c]) ? make_double2(sqrt(fmax(rn2[c].x, 0.0)), 0.0) : make_double2(0, 0);
}

// Back substitution of column blockIdx.x: H_c[0:n_c, 0:n_c] y_c = g_c[0:n_c].
__global__ void __launch_bounds__(kMaxM) many_backsolve_kernel(int m, const int* __restrict__ nstop, const double2* __restrict__ H,
                                                               const double2* __restrict__ g, double2* __restrict__ y)
{
    __shared__ double2 yi;
    const int c = blockIdx.x, t = threadIdx.x, n = nstop[c];
    const double2* Hc = H + (size_t)c * m * (m + 1);
    double2* yc = y + (size_t)c * m;
    double2 gt = t < n ? g[(size_t)c * (m + 1) + t] : make_double2(0, 0);
    for (int i = n - 1; i >= 0; i--) {
        if (t == i) {
            const double2 d = Hc[(size_t)i * (m + 1) + i];
            const double dd = d.x * d.x + d.y * d.y;
            const double2 v = dd > 0 ? make_double2((gt.x * d.x + gt.y * d.y) / dd, (gt.y * d.x - gt.x * d.y) / dd) : make_double2(0, 0);
            yc[i] = v;
            yi = v;
        }
        __syncthreads();
        if (t < i) {
            const double2 p = cmul(Hc[(size_t)i * (m + 1) + t], yi);
            gt.x -= p.x;
            gt.y -= p.y;
        }
        __syncthreads();
    }
}

// x[e] += sum_{k < n_c} Z_k[e] y_c[k] (Z complex128 or complex64, Z_k at Z + k N B).
template <typename C>
__global__ void many_add_zy_kernel(long NB, int B, int m, const C* __restrict__ Z, const int* __restrict__ nstop, const double2* __restrict__ y,
                                   double2* __restrict__ x)
{
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= NB) return;
    const int c = (int)(e % B), n = nstop[c];
    double2 a = x[e];
    for (int k = 0; k < n; k++) {
        const C z = Z[(size_t)k * NB + e];
        const double2 p = cmul(make_double2((double)z.x, (double)z.y), y[(size_t)c * m + k]);
        a.x += p.x;
        a.y += p.y;
    }
    x[e] = a;
}

// Columns c with flag[c] set are zeroed.
__global__ void many_zero_cols_kernel(long NB, int B, const int* __restrict__ flag, double2* __restrict__ x)
{
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e < NB && flag[e % B]) x[e] = make_double2(0, 0);
}

}  // namespace

// Workspace of one operator handle, kept between solves (grown on demand).
struct GmresWork {
    long N = 0;
    int m = 0, nrb = 0;
    double2 *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr, *t = nullptr, *zin = nullptr;
    float2 *V32 = nullptr, *w32 = nullptr;  // mixed precision: complex64 basis and work vector
    double2* vcur = nullptr;                // mixed precision: the current basis vector in complex128
    double2 *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
    double2 *h1 = nullptr, *h2 = nullptr, *part = nullptr, *sc = nullptr;  // sc: scalars (norms^2)
    double* res = nullptr;       // device: |g[j+1]| per step
    double* res_host = nullptr;  // pinned: one slot per step
    unsigned* tickets = nullptr;
    cudaEvent_t ev[2] = {};
    void release()
    {
        for (void* p : {(void*)V, (void*)Z, (void*)w, (void*)r, (void*)t, (void*)zin, (void*)V32, (void*)w32, (void*)vcur, (void*)H, (void*)cs,
                        (void*)sn, (void*)g, (void*)y, (void*)h1, (void*)h2, (void*)part, (void*)sc, (void*)res, (void*)tickets})
            cudaFree(p);
        if (res_host) cudaFreeHost(res_host);
        for (cudaEvent_t& e : ev)
            if (e) cudaEventDestroy(e);
        *this = GmresWork();
    }
};

void gmres_work_free(GmresWork* w)
{
    if (!w) return;
    w->release();
    delete w;
}

namespace {

template <typename P>
void dalloc(P** p, size_t bytes)
{
    if (cudaMalloc((void**)p, bytes) != cudaSuccess) {
        cudaGetLastError();
        fail(DAFMM_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes for GMRES failed");
    }
}

GmresWork& workspace(OpsDev& d, long N, int m)
{
    if (!d.gw) d.gw = new GmresWork();
    GmresWork& W = *d.gw;
    if (W.N == N && W.m >= m) return W;
    W.release();
    W.N = N;
    W.m = m;
    W.nrb = (int)((N + kCR - 1) / kCR);
    dalloc(&W.V, sizeof(double2) * N * (m + 1));
    dalloc(&W.Z, sizeof(double2) * N * m);
    dalloc(&W.w, sizeof(double2) * N);
    dalloc(&W.r, sizeof(double2) * N);
    dalloc(&W.t, sizeof(double2) * N);
    dalloc(&W.zin, sizeof(double2) * N);
    dalloc(&W.V32, sizeof(float2) * N * (m + 1));
    dalloc(&W.w32, sizeof(float2) * N);
    dalloc(&W.vcur, sizeof(double2) * N);
    dalloc(&W.H, sizeof(double2) * (m + 1) * m);
    dalloc(&W.cs, sizeof(double2) * m);
    dalloc(&W.sn, sizeof(double2) * m);
    dalloc(&W.g, sizeof(double2) * (m + 1));
    dalloc(&W.y, sizeof(double2) * m);
    dalloc(&W.h1, sizeof(double2) * (m + 1));
    dalloc(&W.h2, sizeof(double2) * (m + 1));
    dalloc(&W.part, sizeof(double2) * (size_t)W.nrb * (m + 1));
    dalloc(&W.sc, sizeof(double2) * 4);
    dalloc(&W.res, sizeof(double));
    dalloc(&W.tickets, sizeof(unsigned) * 4);
    CK(cudaMemset(W.tickets, 0, sizeof(unsigned) * 4));
    if (cudaMallocHost(&W.res_host, sizeof(double) * (m + 1)) != cudaSuccess) {
        cudaGetLastError();
        fail(DAFMM_ENOMEM, "pinned host allocation for GMRES failed");
    }
    for (cudaEvent_t& e : W.ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    const int tile_max = (int)(sizeof(double2) * kCR * (kMaxM + 1));
    CK(cudaFuncSetAttribute(cgs_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, tile_max));
    CK(cudaFuncSetAttribute(cgs_norm_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, tile_max));
    CK(cudaFuncSetAttribute(cgs_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, tile_max / 2));
    CK(cudaFuncSetAttribute(cgs_norm_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, tile_max / 2));
    return W;
}

// |v|^2 -> *out (real part), no Givens step.
void norm2(GmresWork& W, const double2* v, double2* out, cudaStream_t s)
{
    GivensArgs none{};
    cgs_norm_kernel<double><<<W.nrb, kAT, 0, s>>>(W.N, nullptr, 0, nullptr, (double2*)v, W.part, W.tickets + 3, out, none);
}

}  // namespace

int gmres_run(const Tree& t, OpsDev& d, const void* M, PrecFn prec, const double* f, double* x, const gmres_opts& o, gmres_stats& st,
              cudaStream_t s)
{
    auto t0 = std::chrono::steady_clock::now();
    const long N = t.N;
    const int m = o.restart;
    if (m < 1 || m > kMaxM) fail(DAFMM_EBADARG, "restart must be in 1..128");
    GmresWork& W = workspace(d, N, m);
    double2* X = (double2*)x;
    const double2* F = (const double2*)f;
    auto read_sqrt = [&](const double2* dev) {
        double2 h;
        CK(cudaMemcpyAsync(&h, dev, sizeof(double2), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return std::sqrt(std::max(h.x, 0.0));
    };
    norm2(W, F, W.sc, s);
    const double nf = read_sqrt(W.sc);
    std::memset(&st, 0, sizeof(st));
    if (nf == 0.0) {
        CK(cudaMemsetAsync(X, 0, sizeof(double2) * N, s));
        CK(cudaStreamSynchronize(s));
        st.converged = 1;
        return DAFMM_OK;
    }
    // Mixed precision keeps the inner cycles' basis in complex64 (CGS2 in FP32
    // keeps it orthogonal to ~1e-7, far below the inner tolerance) and the
    // current basis vector in complex128 for the preconditioner; FP64 cycles
    // keep the complex128 basis.  The Hessenberg matrix, the rotations, the
    // preconditioned basis Z and x stay FP64.
    const bool lowp = o.precision == DAFMM_MIXED;
    // one Arnoldi step: v_j -> z_j, w = A z_j, orthogonalise, Givens, v_{j+1}
    // left preconditioning (the paper's M^{-1} A x = M^{-1} f): w = M^{-1} A v_j and
    // x += V y; right preconditioning: z_j = M^{-1} v_j, w = A z_j and x += Z y
    const bool left = prec && o.side == DAFMM_PREC_LEFT;
    auto enqueue_step = [&](int j) {
        const double2* vj = lowp ? W.vcur : W.V + (size_t)j * N;
        if (left) {
            CK(cudaMemcpyAsync(W.zin, vj, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
            apply_matvec(t, d, 1, (const double*)W.zin, (double*)W.t, o.precision, s);
            st.matvecs++;
            prec(M, (const double*)W.t, (double*)W.w, o.precision, s);
            st.precond_applies++;
        } else {
            double2* zj = W.Z + (size_t)j * N;
            if (prec) {
                prec(M, (const double*)vj, (double*)zj, o.precision, s);
                st.precond_applies++;
            } else {
                CK(cudaMemcpyAsync(zj, vj, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
            }
            // fixed buffers keep the captured application valid from one step to the next
            CK(cudaMemcpyAsync(W.zin, zj, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
            apply_matvec(t, d, 1, (const double*)W.zin, (double*)W.w, o.precision, s);
            st.matvecs++;
        }
        // classical Gram-Schmidt, twice; then |w|, the Givens step and v_{j+1}
        GivensArgs gv{j, m, W.h1, W.h2, W.H, W.cs, W.sn, W.g, W.res};
        if (lowp) {
            const size_t tile = sizeof(float2) * kCR * (size_t)(j + 1);
            cgs_kernel<float><<<W.nrb, kAT, tile, s>>>(N, W.V32, j + 1, nullptr, W.w32, W.w, W.part, W.tickets + 0, W.h1);
            cgs_kernel<float><<<W.nrb, kAT, tile, s>>>(N, W.V32, j + 1, W.h1, W.w32, nullptr, W.part, W.tickets + 1, W.h2);
            cgs_norm_kernel<float><<<W.nrb, kAT, tile, s>>>(N, W.V32, j + 1, W.h2, W.w32, W.part, W.tickets + 2, W.sc + 2, gv);
            scale_inv_norm_kernel<float>
                <<<blocks(N), kThreads, 0, s>>>(N, W.w32, nullptr, W.sc + 2, W.V32 + (size_t)(j + 1) * N, W.vcur);
        } else {
            const size_t tile = sizeof(double2) * kCR * (size_t)(j + 1);
            cgs_kernel<double><<<W.nrb, kAT, tile, s>>>(N, W.V, j + 1, nullptr, W.w, nullptr, W.part, W.tickets + 0, W.h1);
            cgs_kernel<double><<<W.nrb, kAT, tile, s>>>(N, W.V, j + 1, W.h1, W.w, nullptr, W.part, W.tickets + 1, W.h2);
            cgs_norm_kernel<double><<<W.nrb, kAT, tile, s>>>(N, W.V, j + 1, W.h2, W.w, W.part, W.tickets + 2, W.sc + 2, gv);
            scale_inv_norm_kernel<double>
                <<<blocks(N), kThreads, 0, s>>>(N, W.w, nullptr, W.sc + 2, W.V + (size_t)(j + 1) * N, nullptr);
        }
        CK(cudaMemcpyAsync(W.res_host + j, W.res, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaEventRecord(W.ev[j & 1], s));
    };
    int total = 0;
    double rel = 0;
    // a zero initial guess needs no application for its residual
    norm2(W, X, W.sc + 3, s);
    bool x_zero = read_sqrt(W.sc + 3) == 0.0;
    for (int outer = 0;; outer++) {
        // true residual in FP64: r = f - A x
        if (x_zero) {
            CK(cudaMemcpyAsync(W.r, F, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
            x_zero = false;
        } else {
            apply_matvec(t, d, 1, (const double*)X, (double*)W.t, DAFMM_FP64, s);
            st.matvecs++;
            sub_kernel<<<blocks(N), kThreads, 0, s>>>(N, F, W.t, W.r);
        }
        norm2(W, W.r, W.sc + 1, s);
        const double rn = read_sqrt(W.sc + 1);
        rel = rn / nf;
        if (o.history && total < o.history_len) o.history[total] = rel;
        st.outer_iterations = outer;
        if (rel <= o.tol) {
            st.converged = 1;
            break;
        }
        if (total >= o.max_iters) break;
        // one flexible GMRES cycle on A d = r (left: M^{-1} A d = M^{-1} r), d0 = 0
        const double inner = o.precision == DAFMM_MIXED ? std::max(o.inner_tol, o.tol / rel * 0.5) : o.tol / rel * 0.5;
        const double2* r0 = W.r;
        double2* r0n2 = W.sc + 1;
        double rn0 = rn;  // norm of the cycle's starting vector
        if (left) {
            prec(M, (const double*)W.r, (double*)W.t, o.precision, s);
            st.precond_applies++;
            norm2(W, W.t, W.sc + 3, s);
            rn0 = read_sqrt(W.sc + 3);
            r0 = W.t;
            r0n2 = W.sc + 3;
        }
        if (lowp)
            scale_inv_norm_kernel<float><<<blocks(N), kThreads, 0, s>>>(N, nullptr, r0, r0n2, W.V32, W.vcur);
        else
            scale_inv_norm_kernel<double><<<blocks(N), kThreads, 0, s>>>(N, nullptr, r0, r0n2, W.V, nullptr);
        init_g_kernel<<<(m + 1 + 127) / 128, 128, 0, s>>>(m, r0n2, W.g);
        const int steps = std::min(m, o.max_iters - total);  // steps this cycle may take
        enqueue_step(0);
        int queued = 1, j = 0;
        double e1 = 1.0, e2 = 1.0;  // the last two estimates (relative to |r|)
        for (;; j++) {
            // queue step j + 1 now if the estimates predict that step j misses the
            // target by far (a needless step costs a full application; waiting
            // costs only the time to queue the next launch)
            if (queued == j + 1 && j + 1 < steps) {
                const double pred = j >= 2 ? e1 * std::min(1.0, e1 / e2) : e1;
                if (pred > 30.0 * inner) {
                    enqueue_step(j + 1);
                    queued++;
                }
            }
            CK(cudaEventSynchronize(W.ev[j & 1]));
            total++;
            const double est = W.res_host[j] / rn0;
            if (o.history && total < o.history_len) o.history[total] = est * rel;
            if (est <= inner || j + 1 >= steps) {
                j++;
                break;
            }
            if (queued == j + 1) {
                enqueue_step(j + 1);
                queued++;
            }
            e2 = e1;
            e1 = est;
        }
        backsolve_kernel<<<1, kMaxM, 0, s>>>(j, m, W.H, W.g, W.y);
        if (!left)
            add_zy_kernel<double2><<<blocks(N), kThreads, 0, s>>>(N, W.Z, N, j, W.y, X);
        else if (lowp)
            add_zy_kernel<float2><<<blocks(N), kThreads, 0, s>>>(N, W.V32, N, j, W.y, X);
        else
            add_zy_kernel<double2><<<blocks(N), kThreads, 0, s>>>(N, W.V, N, j, W.y, X);
        CK(cudaGetLastError());
    }
    CK(cudaStreamSynchronize(s));
    st.iterations = total;
    st.rel_residual = rel;
    st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st.converged ? DAFMM_OK : DAFMM_ENOTCONV;
}


// Workspace of the several-right-hand-side solve (vectors [N][B], bases
// [k][N][B]), kept on the handle and grown on demand.
struct GmresMany {
    long N = 0;
    int B = 0, m = 0, nrb = 0;
    bool v64 = false, v32 = false, z = false;  // which bases are allocated
    double2 *V64 = nullptr, *Z = nullptr, *w64 = nullptr, *r = nullptr, *tv = nullptr, *zin = nullptr, *vcur = nullptr;
    float2 *V32 = nullptr, *w32 = nullptr;
    double2 *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr, *h1 = nullptr, *h2 = nullptr, *part = nullptr,
            *sc = nullptr;  // sc: [4][B] squared column norms
    double* res = nullptr;
    double* res_host = nullptr;
    int *nstop = nullptr, *active = nullptr, *flag = nullptr;
    void release()
    {
        for (void* p : {(void*)V64, (void*)Z, (void*)w64, (void*)r, (void*)tv, (void*)zin, (void*)vcur, (void*)V32, (void*)w32, (void*)H,
                        (void*)cs, (void*)sn, (void*)g, (void*)y, (void*)h1, (void*)h2, (void*)part, (void*)sc, (void*)res, (void*)nstop,
                        (void*)active, (void*)flag})
            cudaFree(p);
        if (res_host) cudaFreeHost(res_host);
        *this = GmresMany();
    }
};

namespace {

GmresMany& many_workspace(GmresMany& W, long N, int B, int m, bool need64, bool need32, bool needZ)
{
    if (!(W.N == N && W.B == B && W.m >= m)) {
        W.release();
        W.N = N;
        W.B = B;
        W.m = m;
        W.nrb = (int)((N + kMRows - 1) / kMRows);
        const size_t NB = (size_t)N * B;
        dalloc(&W.w64, sizeof(double2) * NB);
        dalloc(&W.r, sizeof(double2) * NB);
        dalloc(&W.tv, sizeof(double2) * NB);
        dalloc(&W.zin, sizeof(double2) * NB);
        dalloc(&W.H, sizeof(double2) * B * (size_t)(m + 1) * m);
        dalloc(&W.cs, sizeof(double2) * B * (size_t)m);
        dalloc(&W.sn, sizeof(double2) * B * (size_t)m);
        dalloc(&W.g, sizeof(double2) * B * (size_t)(m + 1));
        dalloc(&W.y, sizeof(double2) * B * (size_t)m);
        dalloc(&W.h1, sizeof(double2) * B * (size_t)(m + 1));
        dalloc(&W.h2, sizeof(double2) * B * (size_t)(m + 1));
        dalloc(&W.part, sizeof(double2) * B * (size_t)(m + 1) * W.nrb);
        dalloc(&W.sc, sizeof(double2) * 4 * B);
        dalloc(&W.res, sizeof(double) * B);
        dalloc(&W.nstop, sizeof(int) * B);
        dalloc(&W.active, sizeof(int) * B);
        dalloc(&W.flag, sizeof(int) * B);
        if (cudaMallocHost(&W.res_host, sizeof(double) * B) != cudaSuccess) {
            cudaGetLastError();
            fail(DAFMM_ENOMEM, "pinned host allocation for GMRES failed");
        }
    }
    const size_t NB = (size_t)N * B;
    if (need64 && !W.v64) {
        dalloc(&W.V64, sizeof(double2) * NB * (W.m + 1));
        W.v64 = true;
    }
    if (need32 && !W.v32) {
        dalloc(&W.V32, sizeof(float2) * NB * (W.m + 1));
        dalloc(&W.w32, sizeof(float2) * NB);
        dalloc(&W.vcur, sizeof(double2) * NB);
        W.v32 = true;
    }
    if (needZ && !W.z) {
        dalloc(&W.Z, sizeof(double2) * NB * W.m);
        W.z = true;
    }
    return W;
}

}  // namespace

void gmres_many_free(GmresMany* w)
{
    if (!w) return;
    w->release();
    delete w;
}

int gmres_run_many(const Tree& t, OpsDev& d, const void* M, PrecManyFn prec, int B, const double* f, double* x, const gmres_opts& o,
                   gmres_stats* st, cudaStream_t s)
{
    auto t0 = std::chrono::steady_clock::now();
    const long N = t.N, NB = N * (long)B;
    const int m = o.restart;
    if (m < 1 || m > kMaxM) fail(DAFMM_EBADARG, "restart must be in 1..128");
    if (B < 2 || B > kMB) fail(DAFMM_EBADARG, "several right-hand sides: 2..64");
    const bool lowp = o.precision == DAFMM_MIXED;
    const bool left = prec && o.side == DAFMM_PREC_LEFT;
    const bool useZ = prec && !left;
    if (!d.gm) d.gm = new GmresMany();
    GmresMany& W = many_workspace(*d.gm, N, B, m, !lowp, lowp, useZ);
    double2* X = (double2*)x;
    const double2* F = (const double2*)f;
    const unsigned nbl = (unsigned)((NB + kThreads - 1) / kThreads);
    std::vector<double2> hb(B);
    // squared column norms of a complex128 [N][B] block into out[0..B)
    auto norms = [&](const double2* v, double2* out) {
        many_dots_kernel<double><<<dim3(W.nrb, 1), kMT, 0, s>>>(N, B, v, 1, v, W.part);
        many_reduce_kernel<<<1, kMT, 0, s>>>(W.nrb, B, W.part, out);
    };
    auto read_norms = [&](const double2* dev, std::vector<double>& out) {
        CK(cudaMemcpyAsync(hb.data(), dev, sizeof(double2) * B, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int c = 0; c < B; c++) out[c] = std::sqrt(std::max(hb[c].x, 0.0));
    };
    auto upload = [&](int* dev, const std::vector<int>& h) {
        CK(cudaMemcpyAsync(dev, h.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
    };
    int matvecs = 0, applies = 0;
    // one lockstep Arnoldi step for every column
    auto enqueue_step = [&](int j) {
        const double2* vj = lowp ? W.vcur : W.V64 + (size_t)j * NB;
        if (left) {
            CK(cudaMemcpyAsync(W.zin, vj, sizeof(double2) * NB, cudaMemcpyDeviceToDevice, s));
            apply_matvec(t, d, B, (const double*)W.zin, (double*)W.tv, o.precision, s);
            matvecs++;
            prec(M, B, (const double*)W.tv, (double*)W.w64, o.precision, s);
            applies++;
        } else {
            if (useZ) {
                double2* zj = W.Z + (size_t)j * NB;
                prec(M, B, (const double*)vj, (double*)zj, o.precision, s);
                applies++;
                CK(cudaMemcpyAsync(W.zin, zj, sizeof(double2) * NB, cudaMemcpyDeviceToDevice, s));
            } else {
                CK(cudaMemcpyAsync(W.zin, vj, sizeof(double2) * NB, cudaMemcpyDeviceToDevice, s));
            }
            apply_matvec(t, d, B, (const double*)W.zin, (double*)W.w64, o.precision, s);
            matvecs++;
        }
        const int nk = j + 1;
        const dim3 gd(W.nrb, (nk + kMK - 1) / kMK);
        double2* wn2 = W.sc + 2 * B;
        if (lowp) {
            many_update_kernel<float><<<nbl, kThreads, 0, s>>>(NB, B, W.V32, 0, nullptr, W.w32, W.w64);
            many_dots_kernel<float><<<gd, kMT, 0, s>>>(N, B, W.V32, nk, W.w32, W.part);
            many_reduce_kernel<<<nk, kMT, 0, s>>>(W.nrb, B, W.part, W.h1);
            many_update_kernel<float><<<nbl, kThreads, 0, s>>>(NB, B, W.V32, nk, W.h1, W.w32, nullptr);
            many_dots_kernel<float><<<gd, kMT, 0, s>>>(N, B, W.V32, nk, W.w32, W.part);
            many_reduce_kernel<<<nk, kMT, 0, s>>>(W.nrb, B, W.part, W.h2);
            many_update_kernel<float><<<nbl, kThreads, 0, s>>>(NB, B, W.V32, nk, W.h2, W.w32, nullptr);
            many_dots_kernel<float><<<dim3(W.nrb, 1), kMT, 0, s>>>(N, B, W.w32, 1, W.w32, W.part);
            many_reduce_kernel<<<1, kMT, 0, s>>>(W.nrb, B, W.part, wn2);
            many_givens_kernel<<<1, kMB, 0, s>>>(j, m, B, W.h1, W.h2, wn2, W.H, W.cs, W.sn, W.g, W.res);
            many_scale_kernel<float><<<nbl, kThreads, 0, s>>>(NB, B, W.w32, nullptr, wn2, W.active, W.V32 + (size_t)(j + 1) * NB, W.vcur);
        } else {
            many_dots_kernel<double><<<gd, kMT, 0, s>>>(N, B, W.V64, nk, W.w64, W.part);
            many_reduce_kernel<<<nk, kMT, 0, s>>>(W.nrb, B, W.part, W.h1);
            many_update_kernel<double><<<nbl, kThreads, 0, s>>>(NB, B, W.V64, nk, W.h1, W.w64, nullptr);
            many_dots_kernel<double><<<gd, kMT, 0, s>>>(N, B, W.V64, nk, W.w64, W.part);
            many_reduce_kernel<<<nk, kMT, 0, s>>>(W.nrb, B, W.part, W.h2);
            many_update_kernel<double><<<nbl, kThreads, 0, s>>>(NB, B, W.V64, nk, W.h2, W.w64, nullptr);
            many_dots_kernel<double><<<dim3(W.nrb, 1), kMT, 0, s>>>(N, B, W.w64, 1, W.w64, W.part);
            many_reduce_kernel<<<1, kMT, 0, s>>>(W.nrb, B, W.part, wn2);
            many_givens_kernel<<<1, kMB, 0, s>>>(j, m, B, W.h1, W.h2, wn2, W.H, W.cs, W.sn, W.g, W.res);
            many_scale_kernel<double>
                <<<nbl, kThreads, 0, s>>>(NB, B, W.w64, nullptr, wn2, W.active, W.V64 + (size_t)(j + 1) * NB, nullptr);
        }
        CK(cudaMemcpyAsync(W.res_host, W.res, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
    };
    std::vector<double> nf(B), rn(B), rn0(B), rel(B, 0.0), inner(B), xn(B);
    std::vector<int> done(B, 0), stop(B, 0), act(B, 0), zf(B, 0), iters(B, 0), outers(B, 0);
    norms(F, W.sc);
    read_norms(W.sc, nf);
    // a zero right-hand side has the zero solution
    bool anyzero = false;
    for (int c = 0; c < B; c++) {
        zf[c] = nf[c] == 0.0;
        anyzero |= zf[c] != 0;
    }
    if (anyzero) {
        upload(W.flag, zf);
        many_zero_cols_kernel<<<nbl, kThreads, 0, s>>>(NB, B, W.flag, X);
    }
    norms(X, W.sc + B);
    read_norms(W.sc + B, xn);
    bool x_zero = true;
    for (int c = 0; c < B; c++) x_zero &= xn[c] == 0.0;
    int total = 0;
    bool all = false;
    for (int outer = 0;; outer++) {
        // true residuals in FP64: r = f - A x (a zero initial guess needs no application)
        if (x_zero) {
            CK(cudaMemcpyAsync(W.r, F, sizeof(double2) * NB, cudaMemcpyDeviceToDevice, s));
            x_zero = false;
        } else {
            apply_matvec(t, d, B, (const double*)X, (double*)W.tv, DAFMM_FP64, s);
            matvecs++;
            sub_kernel<<<nbl, kThreads, 0, s>>>(NB, F, W.tv, W.r);
        }
        norms(W.r, W.sc);
        read_norms(W.sc, rn);
        all = true;
        double worst = 0;
        for (int c = 0; c < B; c++) {
            rel[c] = nf[c] > 0 ? rn[c] / nf[c] : 0.0;
            if (!done[c]) outers[c] = outer;
            done[c] = rel[c] <= o.tol;
            all &= done[c] != 0;
            worst = std::max(worst, rel[c]);
        }
        if (o.history && total < o.history_len) o.history[total] = worst;
        if (all || total >= o.max_iters) break;
        // one flexible GMRES cycle per unfinished column on A d = r (left: M^{-1} A d = M^{-1} r)
        for (int c = 0; c < B; c++) {
            act[c] = !done[c];
            inner[c] = lowp ? std::max(o.inner_tol, o.tol / rel[c] * 0.5) : o.tol / rel[c] * 0.5;
        }
        upload(W.active, act);
        const double2* r0 = W.r;
        double2* r0n2 = W.sc;
        rn0 = rn;
        if (left) {
            prec(M, B, (const double*)W.r, (double*)W.tv, o.precision, s);
            applies++;
            norms(W.tv, W.sc + B);
            read_norms(W.sc + B, rn0);
            r0 = W.tv;
            r0n2 = W.sc + B;
        }
        if (lowp)
            many_scale_kernel<float><<<nbl, kThreads, 0, s>>>(NB, B, nullptr, r0, r0n2, W.active, W.V32, W.vcur);
        else
            many_scale_kernel<double><<<nbl, kThreads, 0, s>>>(NB, B, nullptr, r0, r0n2, W.active, W.V64, nullptr);
        many_init_g_kernel<<<(B * (m + 1) + 127) / 128, 128, 0, s>>>(m, B, r0n2, W.active, W.g);
        const int steps = std::min(m, o.max_iters - total);
        for (int c = 0; c < B; c++) stop[c] = act[c] ? -1 : 0;
        for (int j = 0;; j++) {
            enqueue_step(j);
            CK(cudaStreamSynchronize(s));
            total++;
            bool running = false;
            double mx = 0;
            for (int c = 0; c < B; c++) {
                if (stop[c] >= 0) continue;
                const double est = rn0[c] > 0 ? W.res_host[c] / rn0[c] : 0.0;
                mx = std::max(mx, est * rel[c]);
                if (est <= inner[c])
                    stop[c] = j + 1;
                else
                    running = true;
            }
            if (o.history && total < o.history_len) o.history[total] = mx;
            if (!running) break;
            if (j + 1 >= steps) {
                for (int c = 0; c < B; c++)
                    if (stop[c] < 0) stop[c] = j + 1;
                break;
            }
        }
        for (int c = 0; c < B; c++) iters[c] += stop[c];
        upload(W.nstop, stop);
        many_backsolve_kernel<<<B, kMaxM, 0, s>>>(m, W.nstop, W.H, W.g, W.y);
        if (useZ)
            many_add_zy_kernel<double2><<<nbl, kThreads, 0, s>>>(NB, B, m, W.Z, W.nstop, W.y, X);
        else if (lowp)
            many_add_zy_kernel<float2><<<nbl, kThreads, 0, s>>>(NB, B, m, W.V32, W.nstop, W.y, X);
        else
            many_add_zy_kernel<double2><<<nbl, kThreads, 0, s>>>(NB, B, m, W.V64, W.nstop, W.y, X);
        CK(cudaGetLastError());
    }
    CK(cudaStreamSynchronize(s));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int c = 0; c < B; c++) {
        std::memset(&st[c], 0, sizeof(gmres_stats));
        st[c].iterations = iters[c];
        st[c].outer_iterations = outers[c];
        st[c].matvecs = matvecs;
        st[c].precond_applies = applies;
        st[c].converged = done[c];
        st[c].rel_residual = rel[c];
        st[c].seconds = secs;
    }
    return all ? DAFMM_OK : DAFMM_ENOTCONV;
}

}  // namespace dafmm
