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

struct HodlrDevLevel {
    int r = 0;
    double2 *R64 = nullptr, *Ut64 = nullptr, *S64 = nullptr;
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
    double2* inv64 = nullptr;
    float2* inv32 = nullptr;
    std::vector<dafmm::HodlrDevLevel> dlv;
    void* t_part = nullptr;  // reduction partials (complex128 size): rmax x N/32
    void* s_buf = nullptr;   // s per node and half: 2 rmax x nodes
    void* xw = nullptr;      // complex64 work vector (mixed precision)
    int rmax = 0;
    double seconds = 0;
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

std::vector<double2> to64(const std::vector<cd>& v)
{
    std::vector<double2> o(v.size());
    for (size_t k = 0; k < v.size(); k++) o[k] = make_double2(v[k].real(), v[k].imag());
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

// x_leaf = Inv_leaf b_leaf; one CTA (leaf threads) per leaf; Inv column-major.
template <typename T>
__global__ void leaf_inv_kernel(int leaf, const typename C2<T>::t* __restrict__ inv, const typename C2<T>::t* __restrict__ b,
                                typename C2<T>::t* __restrict__ x)
{
    using C = typename C2<T>::t;
    extern __shared__ unsigned char sm_raw[];
    C* bs = (C*)sm_raw;
    const long base = (long)blockIdx.x * leaf;
    for (int j = threadIdx.x; j < leaf; j += blockDim.x) bs[j] = b[base + j];
    __syncthreads();
    const C* M = inv + (size_t)blockIdx.x * leaf * leaf;
    for (int i = threadIdx.x; i < leaf; i += blockDim.x) {
        T sr = 0, si = 0;
        for (int j = 0; j < leaf; j++) {
            const C m = M[(size_t)j * leaf + i];
            const C v = bs[j];
            sr += m.x * v.x - m.y * v.y;
            si += m.x * v.y + m.y * v.x;
        }
        C o;
        o.x = sr;
        o.y = si;
        x[base + i] = o;
    }
}

// part[q][g] = sum_{i in group g of 32} R[q][i] x[i]  (segments are >= 32 long)
template <typename T>
__global__ void rx_partial_kernel(long N, int r, const typename C2<T>::t* __restrict__ R, const typename C2<T>::t* __restrict__ x,
                                  typename C2<T>::t* __restrict__ part)
{
    using C = typename C2<T>::t;
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    C p;
    p.x = 0;
    p.y = 0;
    if (i < N) p = cmul(R[(size_t)q * N + i], x[i]);
    for (int o = 16; o > 0; o >>= 1) {
        p.x += __shfl_down_sync(0xffffffffu, p.x, o);
        p.y += __shfl_down_sync(0xffffffffu, p.y, o);
    }
    if ((threadIdx.x & 31) == 0 && i < N) part[(size_t)q * (N / 32) + i / 32] = p;
}

// One CTA per node: t = [V12 x2; V21 x1] from the partials, s = S^{-1} t.
template <typename T>
__global__ void node_small_kernel(long N, long n, int r, const typename C2<T>::t* __restrict__ part,
                                  const typename C2<T>::t* __restrict__ S, typename C2<T>::t* __restrict__ s)
{
    using C = typename C2<T>::t;
    extern __shared__ unsigned char sm_raw[];
    C* t = (C*)sm_raw;
    const long node = blockIdx.x;
    const long g0 = node * n / 32, gh = n / 64;  // groups of the node, of one half
    for (int a = threadIdx.x; a < 2 * r; a += blockDim.x) {
        const int q = a < r ? a : a - r;
        const long gs = a < r ? g0 + gh : g0;  // first r: half 2 (V12 x2); last r: half 1 (V21 x1)
        T sr = 0, si = 0;
        for (long g = 0; g < gh; g++) {
            const C p = part[(size_t)q * (N / 32) + gs + g];
            sr += p.x;
            si += p.y;
        }
        t[a].x = sr;
        t[a].y = si;
    }
    __syncthreads();
    const C* Sn = S + (size_t)node * 4 * r * r;
    for (int a = threadIdx.x; a < 2 * r; a += blockDim.x) {
        T sr = 0, si = 0;
        for (int b = 0; b < 2 * r; b++) {
            const C m = Sn[(size_t)a * 2 * r + b];
            sr += m.x * t[b].x - m.y * t[b].y;
            si += m.x * t[b].y + m.y * t[b].x;
        }
        s[(size_t)node * 2 * r + a].x = sr;
        s[(size_t)node * 2 * r + a].y = si;
    }
}

// x[i] -= sum_q Ut[i][q] s[node(i)][half(i)][q]
template <typename T>
__global__ void update_kernel(long N, long n, int r, const typename C2<T>::t* __restrict__ Ut, const typename C2<T>::t* __restrict__ s,
                              typename C2<T>::t* __restrict__ x)
{
    using C = typename C2<T>::t;
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const long node = i / n;
    const int hh = (i - node * n) >= n / 2 ? 1 : 0;
    const C* sv = s + (size_t)node * 2 * r + hh * r;
    const C* u = Ut + (size_t)i * r;
    C a = x[i];
    for (int q = 0; q < r; q++) {
        const C p = cmul(u[q], sv[q]);
        a.x -= p.x;
        a.y -= p.y;
    }
    x[i] = a;
}

__global__ void c128_to_c64(long n, const double2* __restrict__ a, float2* __restrict__ b)
{
    long k = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (k < n) b[k] = make_float2((float)a[k].x, (float)a[k].y);
}
__global__ void c64_to_c128(long n, const float2* __restrict__ a, double2* __restrict__ b)
{
    long k = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (k < n) b[k] = make_double2(a[k].x, a[k].y);
}

template <typename T>
void apply(const dafmm_hodlr& h, const typename C2<T>::t* b, typename C2<T>::t* x, cudaStream_t s)
{
    using C = typename C2<T>::t;
    const long N = h.N;
    const long nleaf = N / h.leaf;
    const C* inv = (const C*)(sizeof(T) == 8 ? (const void*)h.inv64 : (const void*)h.inv32);
    leaf_inv_kernel<T><<<(unsigned)nleaf, std::min(h.leaf, 256), sizeof(C) * h.leaf, s>>>(h.leaf, inv, b, x);
    for (int l = h.H - 1; l >= 0; l--) {
        const HodlrDevLevel& L = h.dlv[l];
        const int r = L.r;
        if (r == 0) continue;
        const long n = N >> l;
        const C* R = (const C*)(sizeof(T) == 8 ? (const void*)L.R64 : (const void*)L.R32);
        const C* Ut = (const C*)(sizeof(T) == 8 ? (const void*)L.Ut64 : (const void*)L.Ut32);
        const C* S = (const C*)(sizeof(T) == 8 ? (const void*)L.S64 : (const void*)L.S32);
        rx_partial_kernel<T><<<dim3((unsigned)((N + 255) / 256), r), 256, 0, s>>>(N, r, R, x, (C*)h.t_part);
        node_small_kernel<T><<<(unsigned)(N / n), 64, sizeof(C) * 2 * r, s>>>(N, n, r, (const C*)h.t_part, S, (C*)h.s_buf);
        update_kernel<T><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, n, r, Ut, (const C*)h.s_buf, x);
    }
}

}  // namespace

const dafmm_tree* hodlr_tree(const dafmm_hodlr* h) { return h->tree; }

void hodlr_apply(const dafmm_hodlr* h, const double* b, double* x, int precision, cudaStream_t s)
{
    cudaGetLastError();
    const long N = h->N;
    if (precision == DAFMM_FP64) {
        apply<double>(*h, (const double2*)b, (double2*)x, s);
    } else {
        float2* w = (float2*)h->xw;
        float2* w2 = w + N;
        c128_to_c64<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, (const double2*)b, w2);
        apply<float>(*h, w2, w, s);
        c64_to_c128<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, w, (double2*)x);
    }
    CK(cudaGetLastError());
}

void hodlr_prec(const void* M, const double* v, double* z, int precision, cudaStream_t s)
{
    hodlr_apply((const dafmm_hodlr*)M, v, z, precision, s);
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
        up(to64(invc), &h->inv64);
        up(to32(invc), &h->inv32);
        h->dlv.assign(H, HodlrDevLevel());
        for (int l = 0; l < H; l++) {
            HodlrDevLevel& D = h->dlv[l];
            const HodlrLevelHost& L = h->lv[l];
            D.r = L.r;
            h->rmax = std::max(h->rmax, L.r);
            up(to64(L.R), &D.R64);
            up(to32(L.R), &D.R32);
            up(to64(L.Ut), &D.Ut64);
            up(to32(L.Ut), &D.Ut32);
            up(to64(L.Sinv), &D.S64);
            up(to32(L.Sinv), &D.S32);
        }
        const size_t np = (size_t)std::max(1, h->rmax) * std::max<long>(N / 32, 1);
        if (cudaMalloc(&h->t_part, sizeof(double2) * np) != cudaSuccess ||
            cudaMalloc(&h->s_buf, sizeof(double2) * 2 * std::max(1, h->rmax) * std::max<long>(N / h->leaf, 1)) != cudaSuccess ||
            cudaMalloc(&h->xw, sizeof(float2) * 2 * N) != cudaSuccess) {
            cudaGetLastError();
            fail(DAFMM_ENOMEM, "device allocation for the HODLR work buffers failed");
        }
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
