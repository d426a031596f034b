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
// Arnoldi (classical Gram-Schmidt applied twice), the Hessenberg matrix, the
// Givens rotations and every vector update stay in FP64 on the device; the
// host reads one residual estimate (8 bytes) per inner iteration to decide
// when to stop.  Dot products use two-phase (deterministic) reductions.
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

constexpr int kRowBlock = 2048;  // rows per partial of a dot product
constexpr int kThreads = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b)  // conj(a) * b
{
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// part[k][rb] = sum_{i in block rb} conj(V[i, k]) w[i], k < nk.
__global__ void __launch_bounds__(kThreads) dots_partial_kernel(long N, const double2* __restrict__ V, long ldv, int nk,
                                                                const double2* __restrict__ w, double2* __restrict__ part, int nrb)
{
    __shared__ double2 sh[kThreads / 32];
    const int rb = blockIdx.x, k = blockIdx.y;
    const long i0 = (long)rb * kRowBlock;
    const long i1 = min(N, i0 + kRowBlock);
    const double2* v = V + (size_t)k * ldv;
    double sr = 0, si = 0;
    for (long i = i0 + threadIdx.x; i < i1; i += kThreads) {
        const double2 p = cconjmul(v[i], w[i]);
        sr += p.x;
        si += p.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_down_sync(0xffffffffu, sr, o);
        si += __shfl_down_sync(0xffffffffu, si, o);
    }
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = make_double2(sr, si);
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = make_double2(0, 0);
        for (int q = 0; q < kThreads / 32; q++) {
            t.x += sh[q].x;
            t.y += sh[q].y;
        }
        part[(size_t)k * nrb + rb] = t;
    }
}

// out[k] (+)= sum_rb part[k][rb] for k < nk, in block order.
__global__ void dots_final_kernel(int nk, int nrb, const double2* __restrict__ part, double2* __restrict__ out, int accumulate)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nk) return;
    double2 t = accumulate ? out[k] : make_double2(0, 0);
    for (int rb = 0; rb < nrb; rb++) {
        t.x += part[(size_t)k * nrb + rb].x;
        t.y += part[(size_t)k * nrb + rb].y;
    }
    out[k] = t;
}

// w[i] -= sum_{k<nk} V[i, k] h[k]
__global__ void __launch_bounds__(kThreads) sub_vh_kernel(long N, const double2* __restrict__ V, long ldv, int nk,
                                                          const double2* __restrict__ h, double2* __restrict__ w)
{
    __shared__ double2 hs[128];
    for (int k = threadIdx.x; k < nk; k += blockDim.x) hs[k] = h[k];
    __syncthreads();
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double2 a = w[i];
    for (int k = 0; k < nk; k++) {
        const double2 p = cmul(V[(size_t)k * ldv + i], hs[k]);
        a.x -= p.x;
        a.y -= p.y;
    }
    w[i] = a;
}

// x[i] += sum_{k<nk} Z[i, k] y[k]
__global__ void __launch_bounds__(kThreads) add_zy_kernel(long N, const double2* __restrict__ Z, long ldz, int nk,
                                                          const double2* __restrict__ y, double2* __restrict__ x)
{
    __shared__ double2 ys[128];
    for (int k = threadIdx.x; k < nk; k += blockDim.x) ys[k] = y[k];
    __syncthreads();
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double2 a = x[i];
    for (int k = 0; k < nk; k++) {
        const double2 p = cmul(Z[(size_t)k * ldz + i], ys[k]);
        a.x += p.x;
        a.y += p.y;
    }
    x[i] = a;
}

// out = a * s where s = 1 / sqrt(re(*nrm2)) (scale by the inverse norm), or out = a - b.
__global__ void scale_inv_norm_kernel(long N, const double2* __restrict__ a, const double2* __restrict__ nrm2, double2* __restrict__ out)
{
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double n = sqrt(nrm2->x);
    const double s = n > 0 ? 1.0 / n : 0.0;
    out[i] = make_double2(a[i].x * s, a[i].y * s);
}

__global__ void sub_kernel(long N, const double2* __restrict__ a, const double2* __restrict__ b, double2* __restrict__ out)
{
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    out[i] = make_double2(a[i].x - b[i].x, a[i].y - b[i].y);
}

// Arnoldi bookkeeping for column j (one thread): h[0..j] from the two Gram-
// Schmidt passes, h[j+1] = |w|; apply the previous rotations, form the new
// one, update g and publish |g[j+1]| (the residual norm of the least-squares
// problem).  H is (m+1) x m column-major.
__global__ void givens_kernel(int j, int m, const double2* __restrict__ h1, const double2* __restrict__ h2,
                              const double2* __restrict__ wn2, double2* __restrict__ H, double2* __restrict__ cs,
                              double2* __restrict__ sn, double2* __restrict__ g, double* __restrict__ res)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double2* col = H + (size_t)j * (m + 1);
    for (int k = 0; k <= j; k++) col[k] = make_double2(h1[k].x + h2[k].x, h1[k].y + h2[k].y);
    col[j + 1] = make_double2(sqrt(wn2->x), 0.0);
    // previous rotations: [c s; -conj(s) c] with real c
    for (int k = 0; k < j; k++) {
        const double c = cs[k].x;
        const double2 s = sn[k];
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

// Back substitution H[0:n,0:n] y = g[0:n] (one thread).
__global__ void backsolve_kernel(int n, int m, const double2* __restrict__ H, const double2* __restrict__ g, double2* __restrict__ y)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = n - 1; i >= 0; i--) {
        double2 t = g[i];
        for (int k = i + 1; k < n; k++) {
            const double2 p = cmul(H[(size_t)k * (m + 1) + i], y[k]);
            t.x -= p.x;
            t.y -= p.y;
        }
        const double2 d = H[(size_t)i * (m + 1) + i];
        const double dd = d.x * d.x + d.y * d.y;
        y[i] = dd > 0 ? make_double2((t.x * d.x + t.y * d.y) / dd, (t.y * d.x - t.x * d.y) / dd) : make_double2(0, 0);
    }
}

// g = [|r|, 0, ..., 0]
__global__ void init_g_kernel(int m, const double2* __restrict__ rn2, double2* __restrict__ g)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= m) g[k] = k == 0 ? make_double2(sqrt(rn2->x), 0.0) : make_double2(0, 0);
}

template <typename P>
void dalloc(P** p, size_t bytes)
{
    if (cudaMalloc((void**)p, bytes) != cudaSuccess) {
        cudaGetLastError();
        fail(DAFMM_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes for GMRES failed");
    }
}

struct Work {
    long N = 0;
    int m = 0, nrb = 0;
    double2 *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr, *t = nullptr, *zin = nullptr;
    double2 *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
    double2 *h1 = nullptr, *h2 = nullptr, *part = nullptr, *sc = nullptr;  // sc: scalars (norms^2)
    double* res = nullptr;
    double* res_host = nullptr;  // pinned
    ~Work()
    {
        for (void* p : {(void*)V, (void*)Z, (void*)w, (void*)r, (void*)t, (void*)zin, (void*)H, (void*)cs, (void*)sn, (void*)g, (void*)y, (void*)h1,
                        (void*)h2, (void*)part, (void*)sc, (void*)res})
            cudaFree(p);
        if (res_host) cudaFreeHost(res_host);
    }
};

unsigned blocks(long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// out[0..nk) = V[:, 0..nk)^H w  (accumulate: out += ...)
void dots(Work& W, const double2* V, long ldv, int nk, const double2* w, double2* out, int accumulate, cudaStream_t s)
{
    dots_partial_kernel<<<dim3(W.nrb, nk), kThreads, 0, s>>>(W.N, V, ldv, nk, w, W.part, W.nrb);
    dots_final_kernel<<<(nk + 127) / 128, 128, 0, s>>>(nk, W.nrb, W.part, out, accumulate);
}

}  // namespace

int gmres_run(const Tree& t, OpsDev& d, const void* M, PrecFn prec, const double* f, double* x, const gmres_opts& o, gmres_stats& st,
              cudaStream_t s)
{
    auto t0 = std::chrono::steady_clock::now();
    const long N = t.N;
    const int m = o.restart;
    Work W;
    W.N = N;
    W.m = m;
    W.nrb = (int)((N + kRowBlock - 1) / kRowBlock);
    dalloc(&W.V, sizeof(double2) * N * (m + 1));
    dalloc(&W.Z, sizeof(double2) * N * m);
    dalloc(&W.w, sizeof(double2) * N);
    dalloc(&W.r, sizeof(double2) * N);
    dalloc(&W.t, sizeof(double2) * N);
    dalloc(&W.zin, sizeof(double2) * N);
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
    if (cudaMallocHost(&W.res_host, sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        fail(DAFMM_ENOMEM, "pinned host allocation for GMRES failed");
    }
    double2* X = (double2*)x;
    const double2* F = (const double2*)f;
    auto norm2 = [&](const double2* v, double2* out) { dots(W, v, N, 1, v, out, 0, s); };
    auto read_sqrt = [&](const double2* dev) {
        double2 h;
        CK(cudaMemcpyAsync(&h, dev, sizeof(double2), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return std::sqrt(std::max(h.x, 0.0));
    };
    norm2(F, W.sc);
    const double nf = read_sqrt(W.sc);
    std::memset(&st, 0, sizeof(st));
    if (nf == 0.0) {
        CK(cudaMemsetAsync(X, 0, sizeof(double2) * N, s));
        CK(cudaStreamSynchronize(s));
        st.converged = 1;
        return DAFMM_OK;
    }
    int total = 0;
    double rel = 0;
    for (int outer = 0;; outer++) {
        // true residual in FP64: r = f - A x
        apply_matvec(t, d, 1, (const double*)X, (double*)W.t, DAFMM_FP64, s);
        st.matvecs++;
        sub_kernel<<<blocks(N), kThreads, 0, s>>>(N, F, W.t, W.r);
        norm2(W.r, W.sc + 1);
        const double rn = read_sqrt(W.sc + 1);
        rel = rn / nf;
        if (o.history && total < o.history_len) o.history[total] = rel;
        st.outer_iterations = outer;
        if (rel <= o.tol) {
            st.converged = 1;
            break;
        }
        if (total >= o.max_iters) break;
        // one flexible GMRES cycle on A d = r, d0 = 0
        const double inner = o.precision == DAFMM_MIXED ? std::max(o.inner_tol, o.tol / rel * 0.5) : o.tol / rel * 0.5;
        scale_inv_norm_kernel<<<blocks(N), kThreads, 0, s>>>(N, W.r, W.sc + 1, W.V);
        init_g_kernel<<<(m + 1 + 127) / 128, 128, 0, s>>>(m, W.sc + 1, W.g);
        int j = 0;
        for (; j < m && total < o.max_iters; j++) {
            double2* vj = W.V + (size_t)j * N;
            double2* zj = W.Z + (size_t)j * N;
            if (prec) {
                prec(M, (const double*)vj, (double*)zj, o.precision, s);
                st.precond_applies++;
            } else {
                CK(cudaMemcpyAsync(zj, vj, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
            }
            // fixed buffers keep the captured application valid from one iteration to the next
            CK(cudaMemcpyAsync(W.zin, zj, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
            apply_matvec(t, d, 1, (const double*)W.zin, (double*)W.w, o.precision, s);
            st.matvecs++;
            // classical Gram-Schmidt, twice
            dots(W, W.V, N, j + 1, W.w, W.h1, 0, s);
            sub_vh_kernel<<<blocks(N), kThreads, 0, s>>>(N, W.V, N, j + 1, W.h1, W.w);
            dots(W, W.V, N, j + 1, W.w, W.h2, 0, s);
            sub_vh_kernel<<<blocks(N), kThreads, 0, s>>>(N, W.V, N, j + 1, W.h2, W.w);
            norm2(W.w, W.sc + 2);
            scale_inv_norm_kernel<<<blocks(N), kThreads, 0, s>>>(N, W.w, W.sc + 2, W.V + (size_t)(j + 1) * N);
            givens_kernel<<<1, 1, 0, s>>>(j, m, W.h1, W.h2, W.sc + 2, W.H, W.cs, W.sn, W.g, W.res);
            CK(cudaMemcpyAsync(W.res_host, W.res, sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            total++;
            const double est = *W.res_host / rn;  // relative to this cycle's |r|
            if (o.history && total < o.history_len) o.history[total] = est * rel;
            if (est <= inner) {
                j++;
                break;
            }
        }
        backsolve_kernel<<<1, 1, 0, s>>>(j, m, W.H, W.g, W.y);
        add_zy_kernel<<<blocks(N), kThreads, 0, s>>>(N, W.Z, N, j, W.y, X);
        CK(cudaGetLastError());
    }
    st.iterations = total;
    st.rel_residual = rel;
    st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st.converged ? DAFMM_OK : DAFMM_ENOTCONV;
}

}  // namespace dafmm
