// Device-built table of the matrix entries of Eq. 13 (or of the point
// kernel of Experiment 1) for every leaf offset of the uniform grid.  On a uniform tree K_ij depends only on the offset between
// the target's and the source's leaves and on (i', j'), so one table per leaf
// level holds every entry (the paper tabulates its near- and far-field
// integrals once per level for the same reason, Section 2.3).
//
//   K(offset, i', j') = beta^2 sum_l Q^+_{l,j'} I_l(t),
//   I_l(t) = int_{[-1,1]^2} (i/4) H0^(1)(kappa beta |t - eta|) b_l(eta) d eta,
//   t = 2 * offset + zeta_{i'}  (target in the source box's reference frame).
//
// Far offsets (max |offset| >= 2): the integrand is smooth on the square and
// a 16 x 16 tensor Gauss-Legendre rule is used.  Near offsets: the square is
// written as the signed sum of the four triangles (t, edge); each triangle is
// mapped to (u, s) with y = t + u (h n + s |h| tau) (h the signed distance
// from t to the edge line, n the outward normal, tau the edge tangent), with
// Jacobian u h |h|, which puts the logarithmic singularity of Y0 at u = 0.
// u is integrated on geometric panels [2^-(k+1), 2^-k], s on panels graded
// away from the foot of the perpendicular (the integrand's complex
// singularities sit at s = +-i); 12-point Gauss-Legendre on every panel.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace dafmm {
namespace {

constexpr int kNp = 10;       // p(p+1)/2 basis functions for p = 4
constexpr int kFarM = 16;     // far tensor rule
constexpr int kNearM = 12;    // per-panel rule of the near rule
constexpr int kUPanels = 36;  // [2^-36, 1] in geometric panels, plus [0, 2^-36]

__constant__ double c_qp[kNp * 16];
__constant__ double c_z[4];
__constant__ double c_fx[kFarM], c_fw[kFarM];
__constant__ double c_nx[kNearM], c_nw[kNearM];

// Gauss-Legendre nodes/weights on [-1,1]: Newton on the Legendre recurrence
// with the derivative from P'_m = m (P_{m-1} - x P_m) / (1 - x^2).
void legendre_rule(int m, double* x, double* w)
{
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < m; i++) {
        double xi = std::cos(pi * (4.0 * i + 3.0) / (4.0 * m + 2.0));
        double d = 0;
        for (int it = 0; it < 60; it++) {
            double pa = 1.0, pb = 0.0;
            for (int k = 1; k <= m; k++) {
                double pc = pb;
                pb = pa;
                pa = ((2.0 * k - 1.0) * xi * pb - (k - 1.0) * pc) / k;
            }
            d = m * (pb - xi * pa) / (1.0 - xi * xi);
            double step = pa / d;
            xi -= step;
            if (std::fabs(step) <= 1e-17) break;
        }
        double pa = 1.0, pb = 0.0;
        for (int k = 1; k <= m; k++) {
            double pc = pb;
            pb = pa;
            pa = ((2.0 * k - 1.0) * xi * pb - (k - 1.0) * pc) / k;
        }
        d = m * (pb - xi * pa) / (1.0 - xi * xi);
        x[i] = xi;
        w[i] = 2.0 / ((1.0 - xi * xi) * d * d);
    }
}

// acc[2l], acc[2l+1] += w * G(r) * b_l(y), G = (i/4)(J0 + i Y0), r = |y - t|
// given by the rule (near the target y - t cancels in floating point)
__device__ __forceinline__ void add_point(double yx, double yy, double r, double kb, double w, double* acc)
{
    double z = kb * r;
    double gr = -0.25 * y0(z) * w;
    double gi = 0.25 * j0(z) * w;
    double Tx[4] = {1.0, yx, 2.0 * yx * yx - 1.0, yx * (4.0 * yx * yx - 3.0)};
    double Ty[4] = {1.0, yy, 2.0 * yy * yy - 1.0, yy * (4.0 * yy * yy - 3.0)};
    int l = 0;
#pragma unroll
    for (int d = 0; d < 4; d++)
#pragma unroll
        for (int a = d; a >= 0; a--) {
            double bv = Tx[a] * Ty[d - a];
            acc[2 * l] += gr * bv;
            acc[2 * l + 1] += gi * bv;
            l++;
        }
}

// Quadrature points (y, weight, |y - t|) over the reference square [-1,1]^2
// for a target t that may lie inside or near it: the square as the signed
// sum of the four triangles (t, edge), each mapped to (u, s) with y = t + u
// (h n + s |h| tau), Jacobian u h |h| and |y - t| = u |h| sqrt(1 + s^2); u
// on geometric panels [2^-(k+1), 2^-k], s on panels graded away from the
// foot of the perpendicular, 12-point Gauss-Legendre on every panel.  The
// CTA's threads split the points; f is called for each point this thread
// owns.
template <class F>
__device__ void near_rule(double tx, double ty, F&& f)
{
    // square [-1,1]^2, counter-clockwise vertices
    const double vx[5] = {-1.0, 1.0, 1.0, -1.0, -1.0};
    const double vy[5] = {-1.0, -1.0, 1.0, 1.0, -1.0};
    for (int e = 0; e < 4; e++) {
        const double ax = vx[e], ay = vy[e], bx = vx[e + 1], by = vy[e + 1];
        const double len = hypot(bx - ax, by - ay);
        const double tux = (bx - ax) / len, tuy = (by - ay) / len;  // tangent
        const double nx = tuy, ny = -tux;                            // outward normal
        const double h = (ax - tx) * nx + (ay - ty) * ny;            // signed distance
        const double ah = fabs(h);
        if (ah < 1e-13) continue;
        const double fx = tx + h * nx, fy = ty + h * ny;             // foot
        const double sa = ((ax - fx) * tux + (ay - fy) * tuy) / ah;
        const double sb = ((bx - fx) * tux + (by - fy) * tuy) / ah;
        // s panel breakpoints: sa, +-2^k (k = 0..40) and 0 inside (sa, sb), sb
        // (targets off the grid may lie very close to an edge line, where |s|
        // reaches 2 / |h|; grid targets never pass 2^10)
        double bp[85];
        int nbp = 0;
        bp[nbp++] = sa;
        {
            double cand[83];
            int nc = 0;
            for (int k = 40; k >= 0; k--) cand[nc++] = -ldexp(1.0, k);
            cand[nc++] = 0.0;
            for (int k = 0; k <= 40; k++) cand[nc++] = ldexp(1.0, k);
            for (int k = 0; k < nc; k++)
                if (cand[k] > sa && cand[k] < sb) bp[nbp++] = cand[k];
        }
        bp[nbp++] = sb;
        const int nsp = nbp - 1;
        const int per_panel = kNearM * kNearM;
        const int items = nsp * (kUPanels + 1) * per_panel;
        for (int q = threadIdx.x; q < items; q += blockDim.x) {
            int pt = q % per_panel;
            int rest = q / per_panel;
            int up = rest % (kUPanels + 1);
            int sp = rest / (kUPanels + 1);
            double u0 = (up == kUPanels) ? 0.0 : ldexp(1.0, -(up + 1));
            double u1 = ldexp(1.0, -up);
            double s0 = bp[sp], s1 = bp[sp + 1];
            int iu = pt % kNearM, is = pt / kNearM;
            double u = 0.5 * (u0 + u1) + 0.5 * (u1 - u0) * c_nx[iu];
            double s = 0.5 * (s0 + s1) + 0.5 * (s1 - s0) * c_nx[is];
            double w = 0.25 * (u1 - u0) * (s1 - s0) * c_nw[iu] * c_nw[is];
            double yx = tx + u * (h * nx + s * ah * tux);
            double yy = ty + u * (h * ny + s * ah * tuy);
            f(yx, yy, w * u * h * ah, u * ah * sqrt(1.0 + s * s));
        }
    }
}

// The 16 x 16 tensor Gauss-Legendre points of the reference square (far
// targets); the CTA's threads split them.
template <class F>
__device__ void far_rule(double tx, double ty, F&& f)
{
    for (int q = threadIdx.x; q < kFarM * kFarM; q += blockDim.x) {
        const int a = q % kFarM, b = q / kFarM;
        f(c_fx[a], c_fx[b], c_fw[a] * c_fw[b], hypot(c_fx[a] - tx, c_fx[b] - ty));
    }
}

// Block-wide sum of the 20 accumulators of every thread; result in sh[0..19].
__device__ void block_reduce20(double* acc, double* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < 2 * kNp; k++) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[warp * 2 * kNp + k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 * kNp) {
        double v = 0;
        for (int w = 0; w < nw; w++) v += sh[w * 2 * kNp + threadIdx.x];
        sh[32 * 2 * kNp + threadIdx.x] = v;
    }
    __syncthreads();
}

// Write K(offset, i', :) = beta^2 Q^+^T I from the reduced integrals.
__device__ void write_row(const double* I, double beta2, double2* out)
{
    if (threadIdx.x < 16) {
        int jp = threadIdx.x;
        double re = 0, im = 0;
        for (int l = 0; l < kNp; l++) {
            re += c_qp[l * 16 + jp] * I[2 * l];
            im += c_qp[l * 16 + jp] * I[2 * l + 1];
        }
        out[jp] = make_double2(beta2 * re, beta2 * im);
    }
}

// One CTA per (far offset, target node).
__global__ void far_table_kernel(int nb, double kb, double beta2, double2* tab)
{
    __shared__ double sh[33 * 2 * kNp];
    const int noff = 2 * nb - 1;
    const long cta = blockIdx.x;
    const int ip = (int)(cta % 16);
    const long off = cta / 16;
    const int dx = (int)(off % noff) - (nb - 1), dy = (int)(off / noff) - (nb - 1);
    if (max(abs(dx), abs(dy)) <= 1) return;  // uniform per CTA: handled by the near kernel
    const double tx = 2.0 * dx + c_z[ip & 3], ty = 2.0 * dy + c_z[ip >> 2];
    double acc[2 * kNp];
#pragma unroll
    for (int k = 0; k < 2 * kNp; k++) acc[k] = 0;
    far_rule(tx, ty, [&](double yx, double yy, double w, double r) { add_point(yx, yy, r, kb, w, acc); });
    block_reduce20(acc, sh);
    write_row(sh + 32 * 2 * kNp, beta2, tab + (off * 16 + ip) * 16);
}

// One CTA per (near offset, target node); near offsets are the 3 x 3 block
// around 0 (clipped to the grid).
__global__ void near_table_kernel(int nb, double kb, double beta2, double2* tab)
{
    __shared__ double sh[33 * 2 * kNp];
    const int noff = 2 * nb - 1;
    const int ip = blockIdx.x % 16;
    const int o9 = blockIdx.x / 16;
    const int dx = o9 % 3 - 1, dy = o9 / 3 - 1;
    if (nb == 1 && (dx || dy)) return;
    const long off = (long)(dy + nb - 1) * noff + (dx + nb - 1);
    const double tx = 2.0 * dx + c_z[ip & 3], ty = 2.0 * dy + c_z[ip >> 2];
    double acc[2 * kNp];
#pragma unroll
    for (int k = 0; k < 2 * kNp; k++) acc[k] = 0;

    near_rule(tx, ty, [&](double yx, double yy, double w, double r) { add_point(yx, yy, r, kb, w, acc); });
    block_reduce20(acc, sh);
    write_row(sh + 32 * 2 * kNp, beta2, tab + (off * 16 + ip) * 16);
}

// Point kernel (Experiment 1's N-body operator): K(offset, i', j') =
// G(x_i', x_j') = (i/4) H0^(1)(kappa beta |t - zeta_j'|), t = 2 offset +
// zeta_i' in the source box's reference frame; zero for i = j.  One thread
// per table entry.
__global__ void point_table_kernel(int nb, double kb, double2* tab)
{
    const long noff = (long)(2 * nb - 1) * (2 * nb - 1);
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= noff * 256) return;
    const int jp = (int)(e & 15), ip = (int)((e >> 4) & 15);
    const long off = e >> 8;
    const int dx = (int)(off % (2 * nb - 1)) - (nb - 1), dy = (int)(off / (2 * nb - 1)) - (nb - 1);
    if (dx == 0 && dy == 0 && ip == jp) {
        tab[e] = make_double2(0.0, 0.0);
        return;
    }
    const double tx = 2.0 * dx + c_z[ip & 3] - c_z[jp & 3], ty = 2.0 * dy + c_z[ip >> 2] - c_z[jp >> 2];
    const double z = kb * hypot(tx, ty);
    tab[e] = make_double2(-0.25 * y0(z), 0.25 * j0(z));
}

// ---------------------------------------------------------------------------
// Field evaluation at arbitrary points (Section 6.1's error function E(x)):
// the interpolant psi(x) = sum_l c_l b_l((x - alpha) / beta) of Eq. 7 on the
// leaf containing x, c = Q^+ psi_vec (zero outside the domain), and the
// volume potential u(x) = int_Omega G(x, y) psi(y) dy = beta^2 sum_B
// int_[-1,1]^2 G(kappa beta |t_B - eta|) psi_B(eta) d eta, t_B = (x -
// alpha_B) / beta, with the near rule for boxes within one box width of x
// and the 16 x 16 rule for the others.

// b_l(x, y), l < 10, in the library's order (total degree, then decreasing a).
__device__ __forceinline__ void basis_eval(double x, double y, double* b)
{
    const double Tx[4] = {1.0, x, 2.0 * x * x - 1.0, x * (4.0 * x * x - 3.0)};
    const double Ty[4] = {1.0, y, 2.0 * y * y - 1.0, y * (4.0 * y * y - 3.0)};
    int l = 0;
#pragma unroll
    for (int d = 0; d < 4; d++)
#pragma unroll
        for (int a = d; a >= 0; a--) b[l++] = Tx[a] * Ty[d - a];
}

// c[leaf][l] = sum_j' Q^+_{l j'} psi[leaf 16 + j'] (Eq. 7's coefficients).
__global__ void field_coef_kernel(long nleaf, const double2* __restrict__ psi, double2* __restrict__ coef)
{
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= nleaf * kNp) return;
    const long leaf = e / kNp;
    const int l = (int)(e % kNp);
    double re = 0, im = 0;
    for (int jp = 0; jp < 16; jp++) {
        const double2 v = psi[leaf * 16 + jp];
        re += c_qp[l * 16 + jp] * v.x;
        im += c_qp[l * 16 + jp] * v.y;
    }
    coef[e] = make_double2(re, im);
}

// Leaf (x, y) of Morton index m (x bit below y bit).
__device__ __forceinline__ void leaf_xy(long m, int& lx, int& ly)
{
    lx = 0;
    ly = 0;
    for (int k = 0; k < 31; k++) {
        lx |= (int)((m >> (2 * k)) & 1) << k;
        ly |= (int)((m >> (2 * k + 1)) & 1) << k;
    }
}

__device__ __forceinline__ long leaf_index(int lx, int ly)
{
    long m = 0;
    for (int k = 0; k < 31; k++) m |= ((long)((lx >> k) & 1) << (2 * k)) | ((long)((ly >> k) & 1) << (2 * k + 1));
    return m;
}

// One CTA per point.
__global__ void field_eval_kernel(long m, const double2* __restrict__ pts, int nb, double x0, double beta, double kb,
                                  const double2* __restrict__ coef, double2* __restrict__ u, double2* __restrict__ psi_at)
{
    __shared__ double sh[2 * 32];
    const double2 X = pts[blockIdx.x];
    double ar = 0.0, ai = 0.0;
    const long nleaf = (long)nb * nb;
    for (long leaf = 0; leaf < nleaf; leaf++) {
        int lx, ly;
        leaf_xy(leaf, lx, ly);
        const double tx = (X.x - (x0 + (2.0 * lx + 1.0) * beta)) / beta;
        const double ty = (X.y - (x0 + (2.0 * ly + 1.0) * beta)) / beta;
        double cr[kNp], ci[kNp];
#pragma unroll
        for (int l = 0; l < kNp; l++) {
            const double2 c = __ldg(&coef[leaf * kNp + l]);
            cr[l] = c.x;
            ci[l] = c.y;
        }
        auto f = [&](double yx, double yy, double w, double r) {
            const double z = kb * r;
            const double gr = -0.25 * y0(z) * w, gi = 0.25 * j0(z) * w;
            double b[kNp];
            basis_eval(yx, yy, b);
            double pr = 0.0, pim = 0.0;
#pragma unroll
            for (int l = 0; l < kNp; l++) {
                pr += cr[l] * b[l];
                pim += ci[l] * b[l];
            }
            ar += gr * pr - gi * pim;
            ai += gr * pim + gi * pr;
        };
        if (fmax(fabs(tx), fabs(ty)) < 3.0)
            near_rule(tx, ty, f);
        else
            far_rule(tx, ty, f);
    }
    // block sum in a fixed order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        ar += __shfl_down_sync(0xffffffffu, ar, o);
        ai += __shfl_down_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) {
        sh[2 * warp] = ar;
        sh[2 * warp + 1] = ai;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sr = 0, si = 0;
        for (int w = 0; w < nw; w++) {
            sr += sh[2 * w];
            si += sh[2 * w + 1];
        }
        u[blockIdx.x] = make_double2(beta * beta * sr, beta * beta * si);
        if (psi_at) {
            const double ex = (X.x - x0) / (2.0 * beta), ey = (X.y - x0) / (2.0 * beta);
            double2 pv = make_double2(0.0, 0.0);
            if (ex >= 0.0 && ey >= 0.0 && ex <= nb && ey <= nb) {
                const int lx = min((int)floor(ex), nb - 1), ly = min((int)floor(ey), nb - 1);
                const long leaf = leaf_index(lx, ly);
                double b[kNp];
                basis_eval((X.x - (x0 + (2.0 * lx + 1.0) * beta)) / beta, (X.y - (x0 + (2.0 * ly + 1.0) * beta)) / beta, b);
                for (int l = 0; l < kNp; l++) {
                    const double2 c = coef[leaf * kNp + l];
                    pv.x += c.x * b[l];
                    pv.y += c.y * b[l];
                }
            }
            psi_at[blockIdx.x] = pv;
        }
    }
}

#define CK(x)                                                                                     \
    do {                                                                                          \
        cudaError_t e_ = (x);                                                                     \
        if (e_ != cudaSuccess) {                                                                  \
            cudaGetLastError(); /* do not leave the error for a later check */                    \
            fail(DAFMM_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_));                   \
        }                                                                                         \
    } while (0)

}  // namespace

double build_entry_table(const Tree& t, EntryTable& out, void* stream_)
{
    cudaStream_t stream = (cudaStream_t)stream_;
    auto t0 = std::chrono::steady_clock::now();
    cudaGetLastError();  // launch checks below must see only this call's errors
    const int p = t.p, nb = t.nb;
    // Q^+ in closed form: first-kind nodes make Q^T Q diagonal,
    // Q^+_{(a,b),(k1,k2)} = T_a(z_k1) T_b(z_k2) / (c_a c_b), c_0 = p, c_a = p/2.
    double z[4], qp[kNp * 16];
    cheb_nodes(p, z);
    {
        int l = 0;
        for (int d = 0; d < p; d++)
            for (int a = d; a >= 0; a--) {
                int b = d - a;
                double ca = a == 0 ? p : p / 2.0, cb = b == 0 ? p : p / 2.0;
                for (int k2 = 0; k2 < p; k2++)
                    for (int k1 = 0; k1 < p; k1++) {
                        double ta = std::cos(a * std::acos(z[k1])), tb = std::cos(b * std::acos(z[k2]));
                        qp[l * 16 + k1 + p * k2] = ta * tb / (ca * cb);
                    }
                l++;
            }
    }
    double fx[kFarM], fw[kFarM], nx[kNearM], nw[kNearM];
    legendre_rule(kFarM, fx, fw);
    legendre_rule(kNearM, nx, nw);
    CK(cudaMemcpyToSymbolAsync(c_qp, qp, sizeof(qp), 0, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyToSymbolAsync(c_z, z, sizeof(z), 0, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyToSymbolAsync(c_fx, fx, sizeof(fx), 0, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyToSymbolAsync(c_fw, fw, sizeof(fw), 0, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyToSymbolAsync(c_nx, nx, sizeof(nx), 0, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyToSymbolAsync(c_nw, nw, sizeof(nw), 0, cudaMemcpyHostToDevice, stream));

    const long noff = (long)(2 * nb - 1) * (2 * nb - 1);
    const size_t bytes = (size_t)noff * 256 * sizeof(double2);
    double2* d_tab = nullptr;
    if (cudaMalloc(&d_tab, bytes) != cudaSuccess) {
        cudaGetLastError();
        fail(DAFMM_ENOMEM, "device allocation of the entry table failed");
    }
    const double kb = t.prm.kappa * t.beta, beta2 = t.beta * t.beta;
    cudaError_t e1 = cudaSuccess;
    if (t.prm.kernel == DAFMM_KERNEL_POINTS) {
        point_table_kernel<<<(unsigned)((noff * 256 + 255) / 256), 256, 0, stream>>>(nb, kb, d_tab);
        e1 = cudaGetLastError();
    } else {
        near_table_kernel<<<9 * 16, 256, 0, stream>>>(nb, kb, beta2, d_tab);
        e1 = cudaGetLastError();
        if (nb >= 3 && e1 == cudaSuccess) {
            far_table_kernel<<<(unsigned)(noff * 16), 256, 0, stream>>>(nb, kb, beta2, d_tab);
            e1 = cudaGetLastError();
        }
    }
    out.nb = nb;
    out.tab.resize((size_t)noff * 256);
    cudaError_t e2 = e1 == cudaSuccess ? cudaMemcpyAsync(out.tab.data(), d_tab, bytes, cudaMemcpyDeviceToHost, stream) : e1;
    cudaError_t e3 = e2 == cudaSuccess ? cudaStreamSynchronize(stream) : e2;
    cudaFree(d_tab);
    if (e3 != cudaSuccess) fail(DAFMM_ECUDA, std::string("entry table kernels: ") + cudaGetErrorString(e3));
    out.lx = &t.leaf_x;
    out.ly = &t.leaf_y;
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

void field_eval(const Tree& t, const double* psi, long m, const double* pts, double* u, double* psi_at, cudaStream_t stream)
{
    cudaGetLastError();
    if (t.p != 4) fail(DAFMM_EBADARG, "field evaluation supports p = 4");
    const long nleaf = (long)t.nb * t.nb;
    double2* coef = nullptr;
    if (cudaMallocAsync((void**)&coef, sizeof(double2) * nleaf * kNp, stream) != cudaSuccess) {
        cudaGetLastError();
        fail(DAFMM_ENOMEM, "device allocation of the interpolation coefficients failed");
    }
    field_coef_kernel<<<(unsigned)((nleaf * kNp + 255) / 256), 256, 0, stream>>>(nleaf, (const double2*)psi, coef);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && m > 0) {
        field_eval_kernel<<<(unsigned)m, 256, 0, stream>>>(m, (const double2*)pts, t.nb, t.x0, t.beta, t.prm.kappa * t.beta, coef,
                                                           (double2*)u, (double2*)psi_at);
        e = cudaGetLastError();
    }
    cudaFreeAsync(coef, stream);
    if (e != cudaSuccess) fail(DAFMM_ECUDA, std::string("field evaluation kernels: ") + cudaGetErrorString(e));
}

}  // namespace dafmm
