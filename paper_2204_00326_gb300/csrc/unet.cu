// Learned initial guess and coarse correction: a convolutional U-Net on the
// tree's node grid (not part of the paper's method; its operator, right-hand
// side and solution are those of Eq. 13).
//
// Network (levels L, base channels c0, c_l = c0 2^l): at each level two 3x3
// convolutions (bias, ReLU); 2x2 average pooling between levels; on the way
// up nearest 2x upsampling, a 3x3 up-convolution (bias, ReLU) and the
// concatenation [skip, up] followed by two 3x3 convolutions; a final 1x1
// convolution (bias, no activation).  Zero padding keeps every level's size.
//
// Data: channel-last (NHWC) BF16 activations, FP32 accumulation, FP32 master
// weights with a BF16 copy for the products, FP32 gradients, Adam.  A view of
// a tensor is (pointer, channel stride per pixel, channel offset): the
// concatenation is one buffer whose halves two convolutions write directly.
// Backward of a convolution: weight gradient by a pixel reduction (atomic
// FP32 accumulation over pixel groups), input gradient as the convolution of
// the output gradient with the flipped, transposed kernel.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "ops.h"

namespace dafmm {
namespace {

#define UCK(x)                                                                                    \
    do {                                                                                          \
        cudaError_t e_ = (x);                                                                     \
        if (e_ != cudaSuccess) {                                                                  \
            cudaGetLastError();                                                                   \
            fail(DAFMM_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_));                   \
        }                                                                                         \
    } while (0)

using bf16 = __nv_bfloat16;

__device__ __forceinline__ float ldf(const float* p) { return *p; }
__device__ __forceinline__ float ldf(const bf16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void stf(float* p, float v) { *p = v; }
__device__ __forceinline__ void stf(bf16* p, float v) { *p = __float2bfloat16(v); }

// Convolution tile: 16 x 8 output pixels, 32 output channels, 8 input
// channels per step; 256 threads, thread = 4 pixels x 4 channels.
constexpr int kTW = 16, kTH = 8, kTC = 32, kCI = 8, kThreads = 256;

// out[b,y,x,co] (+)= act(bias[co] + sum_{ky,kx,ci} in[b, y+ky-R, x+kx-R, ci] w[ky,kx,ci,co])
template <int K, typename Tin, typename Tout>
__global__ void __launch_bounds__(kThreads) conv_kernel(int H, int W, int cin, int cout, const Tin* __restrict__ in, int in_stride,
                                                        int in_off, Tout* __restrict__ out, int out_stride, int out_off,
                                                        const bf16* __restrict__ w, const float* __restrict__ bias, int relu, int accumulate)
{
    constexpr int R = K / 2, SW = kTW + K - 1, SH = kTH + K - 1;
    __shared__ float s_in[kCI * SH * SW];      // [c][sy][sx]
    __shared__ float s_w[K * K * kCI * kTC];   // [tap][c][co]
    const int tiles_x = (W + kTW - 1) / kTW;
    const int tx0 = (blockIdx.x % tiles_x) * kTW, ty0 = (blockIdx.x / tiles_x) * kTH;
    const int co0 = blockIdx.y * kTC;
    const int b = blockIdx.z;
    const int t = threadIdx.x, pg = t & 31, cg = t >> 5;
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int i = 0; i < 4; i++) acc[j][i] = 0.f;
    for (int ci0 = 0; ci0 < cin; ci0 += kCI) {
        for (int e = t; e < kCI * SH * SW; e += kThreads) {
            const int sx = e % SW, q = e / SW, sy = q % SH, c = q / SH;
            const int gx = tx0 + sx - R, gy = ty0 + sy - R, gc = ci0 + c;
            float v = 0.f;
            if (gx >= 0 && gx < W && gy >= 0 && gy < H && gc < cin) v = ldf(in + ((size_t)(b * H + gy) * W + gx) * in_stride + in_off + gc);
            s_in[e] = v;
        }
        for (int e = t; e < K * K * kCI * kTC; e += kThreads) {
            const int co = e % kTC, q = e / kTC, c = q % kCI, tap = q / kCI;
            const int gc = ci0 + c, gco = co0 + co;
            s_w[e] = (gc < cin && gco < cout) ? __bfloat162float(w[((size_t)tap * cin + gc) * cout + gco]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int tap = 0; tap < K * K; tap++) {
            const int ky = tap / K, kx = tap % K;
#pragma unroll 2
            for (int c = 0; c < kCI; c++) {
                float wv[4];
#pragma unroll
                for (int i = 0; i < 4; i++) wv[i] = s_w[(tap * kCI + c) * kTC + cg * 4 + i];
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int p = pg + 32 * j, py = p / kTW, px = p % kTW;
                    const float x = s_in[(c * SH + py + ky) * SW + px + kx];
#pragma unroll
                    for (int i = 0; i < 4; i++) acc[j][i] = fmaf(x, wv[i], acc[j][i]);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int p = pg + 32 * j, gx = tx0 + p % kTW, gy = ty0 + p / kTW;
        if (gx >= W || gy >= H) continue;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int co = co0 + cg * 4 + i;
            if (co >= cout) continue;
            float v = acc[j][i] + (bias ? bias[co] : 0.f);
            if (relu) v = fmaxf(v, 0.f);
            Tout* o = out + ((size_t)(b * H + gy) * W + gx) * out_stride + out_off + co;
            if (accumulate) v += ldf(o);
            stf(o, v);
        }
    }
}

// dw[ky,kx,ci,co] += sum over the pixels of this block's tiles of in[b, y+ky-R, x+kx-R, ci] d[b,y,x,co]
// (d: the gradient before the activation, [pixel][cout]).  Block: 8 input x
// 32 output channels, every tap; grid.y splits the pixel tiles.
template <int K, typename Tin>
__global__ void __launch_bounds__(kThreads) wgrad_kernel(int B, int H, int W, int cin, int cout, const Tin* __restrict__ in, int in_stride,
                                                         int in_off, const float* __restrict__ d, float* __restrict__ dw, int tiles_per_block)
{
    constexpr int R = K / 2, SW = kTW + K - 1, SH = kTH + K - 1;
    __shared__ float s_in[kCI * SH * SW];
    __shared__ float s_d[kTH * kTW * kTC];  // [p][co]
    const int nco = (cout + kTC - 1) / kTC;
    const int ci0 = (blockIdx.x / nco) * kCI, co0 = (blockIdx.x % nco) * kTC;
    const int t = threadIdx.x, co = t & 31, c = t >> 5;
    const int tiles_x = (W + kTW - 1) / kTW, tiles_y = (H + kTH - 1) / kTH, ntiles = B * tiles_x * tiles_y;
    float acc[K * K];
#pragma unroll
    for (int k = 0; k < K * K; k++) acc[k] = 0.f;
    for (int tt = blockIdx.y * tiles_per_block; tt < min(ntiles, (blockIdx.y + 1) * tiles_per_block); tt++) {
        const int b = tt / (tiles_x * tiles_y), r = tt % (tiles_x * tiles_y);
        const int tx0 = (r % tiles_x) * kTW, ty0 = (r / tiles_x) * kTH;
        for (int e = t; e < kCI * SH * SW; e += kThreads) {
            const int sx = e % SW, q = e / SW, sy = q % SH, cc = q / SH;
            const int gx = tx0 + sx - R, gy = ty0 + sy - R, gc = ci0 + cc;
            float v = 0.f;
            if (gx >= 0 && gx < W && gy >= 0 && gy < H && gc < cin) v = ldf(in + ((size_t)(b * H + gy) * W + gx) * in_stride + in_off + gc);
            s_in[e] = v;
        }
        for (int e = t; e < kTH * kTW * kTC; e += kThreads) {
            const int cc = e % kTC, p = e / kTC, gx = tx0 + p % kTW, gy = ty0 + p / kTW, gco = co0 + cc;
            s_d[e] = (gx < W && gy < H && gco < cout) ? d[((size_t)(b * H + gy) * W + gx) * cout + gco] : 0.f;
        }
        __syncthreads();
        for (int p = 0; p < kTH * kTW; p++) {
            const float dv = s_d[p * kTC + co];
            const int py = p / kTW, px = p % kTW;
#pragma unroll
            for (int k = 0; k < K * K; k++) acc[k] = fmaf(s_in[(c * SH + py + k / K) * SW + px + k % K], dv, acc[k]);
        }
        __syncthreads();
    }
    // this block's partial of its weights, slot blockIdx.y (summed in slot order by sum_slots_kernel)
    if (ci0 + c < cin && co0 + co < cout) {
        const size_t nw = (size_t)K * K * cin * cout;
#pragma unroll
        for (int k = 0; k < K * K; k++) dw[(size_t)blockIdx.y * nw + ((size_t)k * cin + ci0 + c) * cout + co0 + co] = acc[k];
    }
}

// The partial of sum_p d[p][co] over this block's pixels, slot blockIdx.x.
__global__ void bgrad_kernel(long npix, int cout, const float* __restrict__ d, float* __restrict__ db)
{
    __shared__ float s[8][33];
    const int co = blockIdx.y * 32 + threadIdx.x;
    float a = 0.f;
    if (co < cout)
        for (long p = blockIdx.x * 8 + threadIdx.y; p < npix; p += (long)gridDim.x * 8) a += d[p * cout + co];
    s[threadIdx.y][threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.y == 0 && co < cout) {
        for (int k = 1; k < 8; k++) a += s[k][threadIdx.x];
        db[(size_t)blockIdx.x * cout + co] = a;
    }
}

// out[i] += sum over slots g < G of part[g n + i], in slot order (gradients
// that do not depend on timing, so training is reproducible run to run).
__global__ void sum_slots_kernel(long n, int G, const float* __restrict__ part, float* __restrict__ out)
{
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float a = 0.f;
    for (int g = 0; g < G; g++) a += part[(size_t)g * n + i];
    out[i] += a;
}

// d[p][c] = g[p, goff + c] * (y[p, yoff + c] > 0): the gradient before a ReLU
__global__ void relu_mask_kernel(long npix, int C, const float* __restrict__ g, int gs, int goff, const bf16* __restrict__ y, int ys,
                                 int yoff, float* __restrict__ d)
{
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= npix * C) return;
    const long p = e / C;
    const int c = (int)(e % C);
    d[e] = __bfloat162float(y[p * ys + yoff + c]) > 0.f ? g[p * gs + goff + c] : 0.f;
}

// 2 x 2 average pooling: out[b,y,x,c] = mean of in[b, 2y+dy, 2x+dx, c]
__global__ void pool_kernel(int B, int Ho, int Wo, int C, const bf16* __restrict__ in, int is, int ioff, bf16* __restrict__ out)
{
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= (long)B * Ho * Wo * C) return;
    const int c = (int)(e % C);
    const long p = e / C;
    const int x = (int)(p % Wo), y = (int)((p / Wo) % Ho), b = (int)(p / ((long)Wo * Ho));
    const int Wi = 2 * Wo;
    float s = 0.f;
    for (int dy = 0; dy < 2; dy++)
        for (int dx = 0; dx < 2; dx++) s += __bfloat162float(in[((size_t)(b * 2 * Ho + 2 * y + dy) * Wi + 2 * x + dx) * is + ioff + c]);
    out[e] = __float2bfloat16(0.25f * s);
}

// gin[b, 2y+dy, 2x+dx, c] += gout[b,y,x,c] / 4
__global__ void pool_back_kernel(int B, int Ho, int Wo, int C, const float* __restrict__ gout, float* __restrict__ gin, int gs, int goff)
{
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= (long)B * Ho * Wo * C) return;
    const int c = (int)(e % C);
    const long p = e / C;
    const int x = (int)(p % Wo), y = (int)((p / Wo) % Ho), b = (int)(p / ((long)Wo * Ho));
    const int Wi = 2 * Wo;
    const float v = 0.25f * gout[e];
    for (int dy = 0; dy < 2; dy++)
        for (int dx = 0; dx < 2; dx++) gin[((size_t)(b * 2 * Ho + 2 * y + dy) * Wi + 2 * x + dx) * gs + goff + c] += v;
}

// nearest 2x upsampling: out[b,y,x,c] = in[b, y/2, x/2, c]
__global__ void up_kernel(int B, int Ho, int Wo, int C, const bf16* __restrict__ in, int is, int ioff, bf16* __restrict__ out)
{
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= (long)B * Ho * Wo * C) return;
    const int c = (int)(e % C);
    const long p = e / C;
    const int x = (int)(p % Wo), y = (int)((p / Wo) % Ho), b = (int)(p / ((long)Wo * Ho));
    out[e] = in[((size_t)(b * (Ho / 2) + y / 2) * (Wo / 2) + x / 2) * is + ioff + c];
}

// gin[b,y,x,c] += sum_{dy,dx} gout[b, 2y+dy, 2x+dx, c]
__global__ void up_back_kernel(int B, int Hi, int Wi, int C, const float* __restrict__ gout, float* __restrict__ gin, int gs, int goff)
{
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= (long)B * Hi * Wi * C) return;
    const int c = (int)(e % C);
    const long p = e / C;
    const int x = (int)(p % Wi), y = (int)((p / Wi) % Hi), b = (int)(p / ((long)Wi * Hi));
    const int Wo = 2 * Wi;
    float s = 0.f;
    for (int dy = 0; dy < 2; dy++)
        for (int dx = 0; dx < 2; dx++) s += gout[((size_t)(b * 2 * Hi + 2 * y + dy) * Wo + 2 * x + dx) * C + c];
    gin[p * gs + goff + c] += s;
}

// wf[ky,kx,co,ci] = w[K-1-ky, K-1-kx, ci, co]: the kernel of the input gradient
__global__ void flip_kernel(int K, int cin, int cout, const bf16* __restrict__ w, bf16* __restrict__ wf)
{
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= (long)K * K * cin * cout) return;
    const int co = (int)(e % cout);
    const long q = e / cout;
    const int ci = (int)(q % cin), tap = (int)(q / cin);
    const int ky = tap / K, kx = tap % K;
    wf[(((size_t)(K - 1 - ky) * K + (K - 1 - kx)) * cout + co) * cin + ci] = w[e];
}

__global__ void to_bf16_kernel(long n, const float* __restrict__ a, bf16* __restrict__ b)
{
    const long k = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (k < n) b[k] = __float2bfloat16(a[k]);
}

// Mean squared error over n outputs: loss += sum (y - t)^2 / n, g = 2 (y - t) / n
__global__ void mse_kernel(long n, const float* __restrict__ y, const float* __restrict__ tg, float* __restrict__ g, double* __restrict__ loss)
{
    __shared__ double s[256];
    double a = 0;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const float d = y[k] - tg[k];
        g[k] = 2.f * d / (float)n;
        a += (double)d * d;
    }
    s[threadIdx.x] = a;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, s[0] / (double)n);
}

// Adam (Kingma & Ba) with bias correction; refreshes the BF16 copy.
__global__ void adam_kernel(long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            bf16* __restrict__ p16, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const long k = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk, vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float pk = p[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    p[k] = pk;
    p16[k] = __float2bfloat16(pk);
}

// Node grid <-> image.  Node n (Morton leaf order, 16 per leaf, k1 + 4 k2)
// sits at pixel (x, y) = (4 lx + k1, 4 ly + k2) of the n_side x n_side image.
__device__ __forceinline__ void node_pixel(long n, int* x, int* y)
{
    const long leaf = n >> 4;
    const int k = (int)(n & 15);
    int lx = 0, ly = 0;
    for (int b = 0; b < 31; b++) {
        lx |= (int)((leaf >> (2 * b)) & 1) << b;
        ly |= (int)((leaf >> (2 * b + 1)) & 1) << b;
    }
    *x = 4 * lx + (k & 3);
    *y = 4 * ly + (k >> 2);
}

// scale[0] = max_n |v_n| (or 1 when v = 0), over N complex entries
__global__ void absmax_kernel(long N, const double2* __restrict__ v, double* __restrict__ scale)
{
    __shared__ double s[256];
    double a = 0;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < N; k += (long)gridDim.x * blockDim.x)
        a = fmax(a, hypot(v[k].x, v[k].y));
    s[threadIdx.x] = a;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax((unsigned long long*)scale, (unsigned long long)__double_as_longlong(s[0]));
}

// image[y, x, :] = (q, Re v / s, Im v / s) of the node at (x, y); s = scale[0] (1 if 0)
__global__ void features_kernel(long N, int side, const double* __restrict__ q, const double2* __restrict__ v,
                                const double* __restrict__ scale, float* __restrict__ img)
{
    const long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= N) return;
    int x, y;
    node_pixel(n, &x, &y);
    const double s = scale[0] > 0 ? scale[0] : 1.0;
    float* o = img + ((size_t)y * side + x) * 3;
    o[0] = (float)q[n];
    o[1] = (float)(v[n].x / s);
    o[2] = (float)(v[n].y / s);
}

// x[n] = a x[n] + c s (out[y, x, 0] + i out[y, x, 1]) at the node's pixel
__global__ void unfeatures_kernel(long N, int side, const float* __restrict__ img, const double* __restrict__ scale, double a, double c,
                                  double2* __restrict__ xv)
{
    const long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= N) return;
    int x, y;
    node_pixel(n, &x, &y);
    const double s = scale[0] > 0 ? scale[0] : 1.0;
    const float* o = img + ((size_t)y * side + x) * 2;
    const double2 old = a != 0 ? xv[n] : make_double2(0, 0);
    xv[n] = make_double2(a * old.x + c * s * o[0], a * old.y + c * s * o[1]);
}

inline unsigned blocks(long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// SplitMix64 (Steele, Lea, Flood 2014) and the Box-Muller transform: the
// weight initialisation's random numbers.
struct Rng {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal()
    {
        const double u = uniform(), v = uniform();
        return std::sqrt(-2.0 * std::log(u)) * std::cos(6.283185307179586 * v);
    }
};

}  // namespace

// ---------------------------------------------------------------------------
// The network and its buffers.
struct UnetConv {
    int cin, cout, K;
    long w_off, b_off;  // in the flat parameter array: weights [K][K][cin][cout], then bias [cout]
};

constexpr int kWSlots = 32;    // pixel-tile slots of a weight-gradient reduction
constexpr int kBSlots = 1024;  // pixel blocks of a bias-gradient reduction

struct UnetAct {
    int B = 0, H = 0, W = 0;
    std::vector<void*> mem;  // every allocation, freed together
    // activations (BF16) and their gradients (FP32), per level
    bf16* x0 = nullptr;
    std::vector<bf16*> ea, cat, pool, up, da, db;
    bf16* eb = nullptr;
    std::vector<float*> gea, gcat, gpool, gup, gda, gdb;
    float* geb = nullptr;
    float* gout = nullptr;  // [pixels][out_ch]
    float* dpre = nullptr;  // scratch: gradient before an activation
    bf16* wflip = nullptr;  // scratch: flipped kernel
    float* wpart = nullptr;  // scratch: per-slot partial weight gradients of one convolution
    float* bpart = nullptr;  // scratch: per-block partial bias gradients
    size_t grad_bytes = 0;  // of the FP32 gradient block (zeroed per backward pass)
    float* grad_block = nullptr;
};

}  // namespace dafmm

struct dafmm_unet {
    unet_params prm{};
    std::vector<dafmm::UnetConv> convs;
    long nparam = 0;
    float* p32 = nullptr;
    dafmm::bf16* p16 = nullptr;
    float* grad = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    long step = 0;
    double* scal = nullptr;   // device scalars: [0] loss, [1] input scale
    float* img_in = nullptr;  // single-image buffers of the guess path
    float* img_out = nullptr;
    long img_pixels = 0;
    dafmm::UnetAct act;
};

namespace dafmm {
namespace {

int ch(const dafmm_unet* u, int l) { return u->prm.base << l; }
int conv_enc(int l, int ab) { return 2 * l + ab; }
int conv_dec(const dafmm_unet* u, int l, int uab) { return 2 * u->prm.levels + 3 * (u->prm.levels - 2 - l) + uab; }
int conv_out(const dafmm_unet* u) { return 2 * u->prm.levels + 3 * (u->prm.levels - 1); }

void act_free(UnetAct& a)
{
    for (void* p : a.mem) cudaFree(p);
    a = UnetAct();
}

template <typename T>
T* act_alloc(UnetAct& a, size_t n)
{
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        fail(DAFMM_ENOMEM, "device allocation for the U-Net activations failed");
    }
    a.mem.push_back(p);
    return (T*)p;
}

// Activations and gradients for batch B of H x W images.
void act_ensure(dafmm_unet* u, int B, int H, int W)
{
    UnetAct& a = u->act;
    if (a.B == B && a.H == H && a.W == W) return;
    act_free(a);
    a.B = B;
    a.H = H;
    a.W = W;
    const int L = u->prm.levels;
    auto px = [&](int l) { return (size_t)B * (H >> l) * (W >> l); };
    a.x0 = act_alloc<bf16>(a, px(0) * u->prm.in_ch);
    a.ea.assign(L, nullptr);
    a.cat.assign(L, nullptr);
    a.pool.assign(L, nullptr);
    a.up.assign(L, nullptr);
    a.da.assign(L, nullptr);
    a.db.assign(L, nullptr);
    for (int l = 0; l < L; l++) {
        a.ea[l] = act_alloc<bf16>(a, px(l) * ch(u, l));
        if (l < L - 1) {
            a.cat[l] = act_alloc<bf16>(a, px(l) * 2 * ch(u, l));
            a.pool[l] = act_alloc<bf16>(a, px(l + 1) * ch(u, l));
            a.up[l] = act_alloc<bf16>(a, px(l) * ch(u, l + 1));
            a.da[l] = act_alloc<bf16>(a, px(l) * ch(u, l));
            a.db[l] = act_alloc<bf16>(a, px(l) * ch(u, l));
        }
    }
    a.eb = act_alloc<bf16>(a, px(L - 1) * ch(u, L - 1));
    // gradients: one block, zeroed per backward pass
    size_t n = 0;
    std::vector<size_t> sz;
    auto add = [&](size_t k) {
        sz.push_back(k);
        n += (k + 63) / 64 * 64;
    };
    for (int l = 0; l < L; l++) {
        add(px(l) * ch(u, l));  // ea
        if (l < L - 1) {
            add(px(l) * 2 * ch(u, l));  // cat
            add(px(l + 1) * ch(u, l));  // pool
            add(px(l) * ch(u, l + 1));  // up
            add(px(l) * ch(u, l));      // da
            add(px(l) * ch(u, l));      // db
        }
    }
    add(px(L - 1) * ch(u, L - 1));  // eb
    a.grad_block = act_alloc<float>(a, n);
    a.grad_bytes = n * sizeof(float);
    float* g = a.grad_block;
    size_t k = 0;
    auto take = [&]() {
        float* r = g;
        g += (sz[k] + 63) / 64 * 64;
        k++;
        return r;
    };
    a.gea.assign(L, nullptr);
    a.gcat.assign(L, nullptr);
    a.gpool.assign(L, nullptr);
    a.gup.assign(L, nullptr);
    a.gda.assign(L, nullptr);
    a.gdb.assign(L, nullptr);
    for (int l = 0; l < L; l++) {
        a.gea[l] = take();
        if (l < L - 1) {
            a.gcat[l] = take();
            a.gpool[l] = take();
            a.gup[l] = take();
            a.gda[l] = take();
            a.gdb[l] = take();
        }
    }
    a.geb = take();
    a.gout = act_alloc<float>(a, px(0) * u->prm.out_ch);
    size_t dpre = 0, wf = 0;
    for (const UnetConv& c : u->convs) wf = std::max(wf, (size_t)c.K * c.K * c.cin * c.cout);
    for (int l = 0; l < L; l++) dpre = std::max(dpre, px(l) * 2 * ch(u, l));
    dpre = std::max(dpre, px(0) * (size_t)std::max(u->prm.out_ch, u->prm.in_ch));
    a.dpre = act_alloc<float>(a, dpre);
    a.wflip = act_alloc<bf16>(a, wf);
    size_t cmax = 1;
    for (const UnetConv& c : u->convs) cmax = std::max(cmax, (size_t)c.cout);
    a.wpart = act_alloc<float>(a, wf * kWSlots);
    a.bpart = act_alloc<float>(a, cmax * kBSlots);
}

template <typename Tin, typename Tout>
void conv(const dafmm_unet* u, int idx, int B, int H, int W, const Tin* in, int is, int ioff, Tout* out, int os, int ooff, bool relu,
          bool accumulate, cudaStream_t s, const bf16* wover = nullptr, bool with_bias = true, int cin = -1, int cout = -1)
{
    const UnetConv& c = u->convs[idx];
    const int ci = cin < 0 ? c.cin : cin, co = cout < 0 ? c.cout : cout;
    const bf16* w = wover ? wover : u->p16 + c.w_off;
    const float* bias = with_bias ? u->p32 + c.b_off : nullptr;
    dim3 grid((unsigned)(((W + kTW - 1) / kTW) * ((H + kTH - 1) / kTH)), (unsigned)((co + kTC - 1) / kTC), (unsigned)B);
    if (c.K == 3)
        conv_kernel<3, Tin, Tout><<<grid, kThreads, 0, s>>>(H, W, ci, co, in, is, ioff, out, os, ooff, w, bias, relu, accumulate);
    else
        conv_kernel<1, Tin, Tout><<<grid, kThreads, 0, s>>>(H, W, ci, co, in, is, ioff, out, os, ooff, w, bias, relu, accumulate);
    UCK(cudaGetLastError());
}

// Weight and bias gradients of conv idx from its input and d (before the activation).
template <typename Tin>
void wgrad(dafmm_unet* u, int idx, int B, int H, int W, const Tin* in, int is, int ioff, const float* d, cudaStream_t s)
{
    const UnetConv& c = u->convs[idx];
    const int ntiles = B * ((W + kTW - 1) / kTW) * ((H + kTH - 1) / kTH);
    const int per = std::max(1, (ntiles + kWSlots - 1) / kWSlots);
    const int G = (ntiles + per - 1) / per;  // slots, at most kWSlots
    const long nw = (long)c.K * c.K * c.cin * c.cout;
    dim3 grid((unsigned)(((c.cin + kCI - 1) / kCI) * ((c.cout + kTC - 1) / kTC)), (unsigned)G);
    if (c.K == 3)
        wgrad_kernel<3, Tin><<<grid, kThreads, 0, s>>>(B, H, W, c.cin, c.cout, in, is, ioff, d, u->act.wpart, per);
    else
        wgrad_kernel<1, Tin><<<grid, kThreads, 0, s>>>(B, H, W, c.cin, c.cout, in, is, ioff, d, u->act.wpart, per);
    sum_slots_kernel<<<blocks(nw), 256, 0, s>>>(nw, G, u->act.wpart, u->grad + c.w_off);
    const long npix = (long)B * H * W;
    const int nbb = (int)std::min<long>(kBSlots, (npix + 7) / 8);
    bgrad_kernel<<<dim3((unsigned)nbb, (unsigned)((c.cout + 31) / 32)), dim3(32, 8), 0, s>>>(npix, c.cout, d, u->act.bpart);
    sum_slots_kernel<<<blocks(c.cout), 256, 0, s>>>(c.cout, nbb, u->act.bpart, u->grad + c.b_off);
    UCK(cudaGetLastError());
}

// gin (+)= conv of d with the flipped, transposed kernel of conv idx.
void dgrad(dafmm_unet* u, int idx, int B, int H, int W, const float* d, float* gin, int gs, int goff, cudaStream_t s)
{
    const UnetConv& c = u->convs[idx];
    const long nw = (long)c.K * c.K * c.cin * c.cout;
    flip_kernel<<<blocks(nw), 256, 0, s>>>(c.K, c.cin, c.cout, u->p16 + c.w_off, u->act.wflip);
    UCK(cudaGetLastError());
    conv<float, float>(u, idx, B, H, W, d, c.cout, 0, gin, gs, goff, false, true, s, u->act.wflip, false, c.cout, c.cin);
}

void relu_mask(long npix, int C, const float* g, int gs, int goff, const bf16* y, int ys, int yoff, float* d, cudaStream_t s)
{
    relu_mask_kernel<<<blocks(npix * C), 256, 0, s>>>(npix, C, g, gs, goff, y, ys, yoff, d);
    UCK(cudaGetLastError());
}

}  // namespace

// ---------------------------------------------------------------------------
dafmm_unet* unet_new(const unet_params& p)
{
    if (p.levels < 1 || p.levels > 6 || p.base < 1 || p.base > 256 || p.in_ch != 3 || p.out_ch != 2)
        fail(DAFMM_EBADARG, "unet_params: levels 1..6, base 1..256, in_ch 3, out_ch 2");
    auto* u = new dafmm_unet();
    u->prm = p;
    const int L = p.levels;
    auto add = [&](int cin, int cout, int K) {
        UnetConv c{cin, cout, K, u->nparam, 0};
        u->nparam += (long)K * K * cin * cout;
        c.b_off = u->nparam;
        u->nparam += cout;
        u->convs.push_back(c);
    };
    for (int l = 0; l < L; l++) {
        add(l == 0 ? p.in_ch : ch(u, l - 1), ch(u, l), 3);
        add(ch(u, l), ch(u, l), 3);
    }
    for (int l = L - 2; l >= 0; l--) {
        add(ch(u, l + 1), ch(u, l), 3);
        add(2 * ch(u, l), ch(u, l), 3);
        add(ch(u, l), ch(u, l), 3);
    }
    add(ch(u, 0), p.out_ch, 1);
    try {
        auto dal = [&](auto** ptr, size_t bytes) {
            if (cudaMalloc((void**)ptr, bytes) != cudaSuccess) {
                cudaGetLastError();
                fail(DAFMM_ENOMEM, "device allocation for the U-Net parameters failed");
            }
        };
        dal(&u->p32, sizeof(float) * u->nparam);
        dal(&u->p16, sizeof(bf16) * u->nparam);
        dal(&u->grad, sizeof(float) * u->nparam);
        dal(&u->m, sizeof(float) * u->nparam);
        dal(&u->v, sizeof(float) * u->nparam);
        dal(&u->scal, sizeof(double) * 4);
        // He initialisation of the weights, zero biases
        std::vector<float> h(u->nparam, 0.f);
        Rng rng{p.seed};
        for (const UnetConv& c : u->convs) {
            const double sd = std::sqrt(2.0 / ((double)c.K * c.K * c.cin));
            for (long k = 0; k < (long)c.K * c.K * c.cin * c.cout; k++) h[c.w_off + k] = (float)(sd * rng.normal());
        }
        unet_set(u, h.data());
        UCK(cudaMemset(u->grad, 0, sizeof(float) * u->nparam));
        UCK(cudaMemset(u->m, 0, sizeof(float) * u->nparam));
        UCK(cudaMemset(u->v, 0, sizeof(float) * u->nparam));
    } catch (...) {
        unet_delete(u);
        throw;
    }
    return u;
}

void unet_delete(dafmm_unet* u)
{
    if (!u) return;
    act_free(u->act);
    cudaFree(u->p32);
    cudaFree(u->p16);
    cudaFree(u->grad);
    cudaFree(u->m);
    cudaFree(u->v);
    cudaFree(u->scal);
    cudaFree(u->img_in);
    cudaFree(u->img_out);
    delete u;
}

long unet_size(const dafmm_unet* u) { return u->nparam; }

void unet_get(const dafmm_unet* u, float* host)
{
    UCK(cudaMemcpy(host, u->p32, sizeof(float) * u->nparam, cudaMemcpyDeviceToHost));
}

void unet_set(dafmm_unet* u, const float* host)
{
    UCK(cudaMemcpy(u->p32, host, sizeof(float) * u->nparam, cudaMemcpyHostToDevice));
    to_bf16_kernel<<<blocks(u->nparam), 256>>>(u->nparam, u->p32, u->p16);
    UCK(cudaGetLastError());
    UCK(cudaDeviceSynchronize());
}

void unet_get_grad(const dafmm_unet* u, float* host)
{
    UCK(cudaMemcpy(host, u->grad, sizeof(float) * u->nparam, cudaMemcpyDeviceToHost));
}

void unet_fwd(dafmm_unet* u, int B, int H, int W, const float* in, float* out, cudaStream_t s)
{
    const int L = u->prm.levels;
    if (B < 1 || H < 1 || W < 1 || H % (1 << (L - 1)) || W % (1 << (L - 1)))
        fail(DAFMM_EBADARG, "unet: batch >= 1 and image sides multiples of 2^(levels-1)");
    act_ensure(u, B, H, W);
    UnetAct& a = u->act;
    const long np0 = (long)B * H * W;
    to_bf16_kernel<<<blocks(np0 * u->prm.in_ch), 256, 0, s>>>(np0 * u->prm.in_ch, in, a.x0);
    UCK(cudaGetLastError());
    for (int l = 0; l < L; l++) {
        const int Hl = H >> l, Wl = W >> l, c = ch(u, l);
        if (l == 0)
            conv<bf16, bf16>(u, conv_enc(l, 0), B, Hl, Wl, a.x0, u->prm.in_ch, 0, a.ea[l], c, 0, true, false, s);
        else
            conv<bf16, bf16>(u, conv_enc(l, 0), B, Hl, Wl, a.pool[l - 1], ch(u, l - 1), 0, a.ea[l], c, 0, true, false, s);
        if (l < L - 1) {
            conv<bf16, bf16>(u, conv_enc(l, 1), B, Hl, Wl, a.ea[l], c, 0, a.cat[l], 2 * c, 0, true, false, s);
            const long n = (long)B * (Hl / 2) * (Wl / 2) * c;
            pool_kernel<<<blocks(n), 256, 0, s>>>(B, Hl / 2, Wl / 2, c, a.cat[l], 2 * c, 0, a.pool[l]);
            UCK(cudaGetLastError());
        } else {
            conv<bf16, bf16>(u, conv_enc(l, 1), B, Hl, Wl, a.ea[l], c, 0, a.eb, c, 0, true, false, s);
        }
    }
    for (int l = L - 2; l >= 0; l--) {
        const int Hl = H >> l, Wl = W >> l, c = ch(u, l), cb = ch(u, l + 1);
        const bf16* below = l + 1 == L - 1 ? a.eb : a.db[l + 1];
        const long n = (long)B * Hl * Wl * cb;
        up_kernel<<<blocks(n), 256, 0, s>>>(B, Hl, Wl, cb, below, cb, 0, a.up[l]);
        UCK(cudaGetLastError());
        conv<bf16, bf16>(u, conv_dec(u, l, 0), B, Hl, Wl, a.up[l], cb, 0, a.cat[l], 2 * c, c, true, false, s);
        conv<bf16, bf16>(u, conv_dec(u, l, 1), B, Hl, Wl, a.cat[l], 2 * c, 0, a.da[l], c, 0, true, false, s);
        conv<bf16, bf16>(u, conv_dec(u, l, 2), B, Hl, Wl, a.da[l], c, 0, a.db[l], c, 0, true, false, s);
    }
    const bf16* top = L == 1 ? a.eb : a.db[0];
    conv<bf16, float>(u, conv_out(u), B, H, W, top, ch(u, 0), 0, out, u->prm.out_ch, 0, false, false, s);
}

double unet_bwd(dafmm_unet* u, int B, int H, int W, const float* in, const float* target, float* out, cudaStream_t s)
{
    const int L = u->prm.levels;
    unet_fwd(u, B, H, W, in, out, s);
    UnetAct& a = u->act;
    const long np0 = (long)B * H * W;
    UCK(cudaMemsetAsync(u->scal, 0, sizeof(double), s));
    UCK(cudaMemsetAsync(u->grad, 0, sizeof(float) * u->nparam, s));
    UCK(cudaMemsetAsync(a.grad_block, 0, a.grad_bytes, s));
    const long nout = np0 * u->prm.out_ch;
    mse_kernel<<<(unsigned)std::min<long>(1024, blocks(nout)), 256, 0, s>>>(nout, out, target, a.gout, u->scal);
    UCK(cudaGetLastError());
    const int c0 = ch(u, 0);
    const bf16* top = L == 1 ? a.eb : a.db[0];
    float* gtop = L == 1 ? a.geb : a.gdb[0];
    wgrad<bf16>(u, conv_out(u), B, H, W, top, c0, 0, a.gout, s);
    dgrad(u, conv_out(u), B, H, W, a.gout, gtop, c0, 0, s);
    for (int l = 0; l <= L - 2; l++) {
        const int Hl = H >> l, Wl = W >> l, c = ch(u, l), cb = ch(u, l + 1);
        const long npx = (long)B * Hl * Wl;
        relu_mask(npx, c, a.gdb[l], c, 0, a.db[l], c, 0, a.dpre, s);
        wgrad<bf16>(u, conv_dec(u, l, 2), B, Hl, Wl, a.da[l], c, 0, a.dpre, s);
        dgrad(u, conv_dec(u, l, 2), B, Hl, Wl, a.dpre, a.gda[l], c, 0, s);
        relu_mask(npx, c, a.gda[l], c, 0, a.da[l], c, 0, a.dpre, s);
        wgrad<bf16>(u, conv_dec(u, l, 1), B, Hl, Wl, a.cat[l], 2 * c, 0, a.dpre, s);
        dgrad(u, conv_dec(u, l, 1), B, Hl, Wl, a.dpre, a.gcat[l], 2 * c, 0, s);
        relu_mask(npx, c, a.gcat[l], 2 * c, c, a.cat[l], 2 * c, c, a.dpre, s);
        wgrad<bf16>(u, conv_dec(u, l, 0), B, Hl, Wl, a.up[l], cb, 0, a.dpre, s);
        dgrad(u, conv_dec(u, l, 0), B, Hl, Wl, a.dpre, a.gup[l], cb, 0, s);
        float* gbelow = l + 1 == L - 1 ? a.geb : a.gdb[l + 1];
        const long n = (long)B * (Hl / 2) * (Wl / 2) * cb;
        up_back_kernel<<<blocks(n), 256, 0, s>>>(B, Hl / 2, Wl / 2, cb, a.gup[l], gbelow, cb, 0);
        UCK(cudaGetLastError());
    }
    for (int l = L - 1; l >= 0; l--) {
        const int Hl = H >> l, Wl = W >> l, c = ch(u, l);
        const long npx = (long)B * Hl * Wl;
        if (l < L - 1) {
            const long n = (long)B * (Hl / 2) * (Wl / 2) * c;
            pool_back_kernel<<<blocks(n), 256, 0, s>>>(B, Hl / 2, Wl / 2, c, a.gpool[l], a.gcat[l], 2 * c, 0);
            UCK(cudaGetLastError());
            relu_mask(npx, c, a.gcat[l], 2 * c, 0, a.cat[l], 2 * c, 0, a.dpre, s);
        } else {
            relu_mask(npx, c, a.geb, c, 0, a.eb, c, 0, a.dpre, s);
        }
        wgrad<bf16>(u, conv_enc(l, 1), B, Hl, Wl, a.ea[l], c, 0, a.dpre, s);
        dgrad(u, conv_enc(l, 1), B, Hl, Wl, a.dpre, a.gea[l], c, 0, s);
        relu_mask(npx, c, a.gea[l], c, 0, a.ea[l], c, 0, a.dpre, s);
        if (l == 0) {
            wgrad<bf16>(u, conv_enc(l, 0), B, Hl, Wl, a.x0, u->prm.in_ch, 0, a.dpre, s);
        } else {
            const int cp = ch(u, l - 1);
            wgrad<bf16>(u, conv_enc(l, 0), B, Hl, Wl, a.pool[l - 1], cp, 0, a.dpre, s);
            dgrad(u, conv_enc(l, 0), B, Hl, Wl, a.dpre, a.gpool[l - 1], cp, 0, s);
        }
    }
    double loss = 0;
    UCK(cudaMemcpyAsync(&loss, u->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    UCK(cudaStreamSynchronize(s));
    return loss;
}

void unet_adam_step(dafmm_unet* u, float lr, float b1, float b2, float eps, cudaStream_t s)
{
    if (!(lr > 0) || !(b1 >= 0 && b1 < 1) || !(b2 >= 0 && b2 < 1) || !(eps > 0)) fail(DAFMM_EBADARG, "adam: lr > 0, 0 <= beta < 1, eps > 0");
    u->step++;
    const float c1 = 1.f - std::pow(b1, (float)u->step), c2 = 1.f - std::pow(b2, (float)u->step);
    adam_kernel<<<blocks(u->nparam), 256, 0, s>>>(u->nparam, u->p32, u->grad, u->m, u->v, u->p16, lr, b1, b2, eps, c1, c2);
    UCK(cudaGetLastError());
}

// x = a x + c s N(q, v / s) on the tree's node grid, s = max |v|.
void unet_apply_nodes(dafmm_unet* u, const Tree& t, const OpsDev& d, const double* v, double* x, double a, double c, cudaStream_t s)
{
    const int side = t.n_side;
    const long N = t.N;
    if ((long)side * side != N) fail(DAFMM_EBADARG, "unet: the tree's nodes do not form a square grid");
    if (u->img_pixels < N) {
        cudaFree(u->img_in);
        cudaFree(u->img_out);
        u->img_in = u->img_out = nullptr;
        u->img_pixels = 0;
        if (cudaMalloc(&u->img_in, sizeof(float) * 3 * N) != cudaSuccess || cudaMalloc(&u->img_out, sizeof(float) * 2 * N) != cudaSuccess) {
            cudaGetLastError();
            fail(DAFMM_ENOMEM, "device allocation for the U-Net images failed");
        }
        u->img_pixels = N;
    }
    UCK(cudaMemsetAsync(u->scal + 1, 0, sizeof(double), s));
    absmax_kernel<<<(unsigned)std::min<long>(1024, blocks(N)), 256, 0, s>>>(N, (const double2*)v, u->scal + 1);
    features_kernel<<<blocks(N), 256, 0, s>>>(N, side, d.q, (const double2*)v, u->scal + 1, u->img_in);
    UCK(cudaGetLastError());
    unet_fwd(u, 1, side, side, u->img_in, u->img_out, s);
    unfeatures_kernel<<<blocks(N), 256, 0, s>>>(N, side, u->img_out, u->scal + 1, a, c, (double2*)x);
    UCK(cudaGetLastError());
}

}  // namespace dafmm

namespace dafmm {
namespace {

// out[0] += sum |f - Ax|^2, out[1] += sum |f|^2
__global__ void resid_kernel(long N, const double2* __restrict__ f, const double2* __restrict__ ax, double* __restrict__ out)
{
    __shared__ double s[2][256];
    double a = 0, b = 0;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < N; k += (long)gridDim.x * blockDim.x) {
        const double rx = f[k].x - ax[k].x, ry = f[k].y - ax[k].y;
        a += rx * rx + ry * ry;
        b += f[k].x * f[k].x + f[k].y * f[k].y;
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s[0][threadIdx.x] += s[0][threadIdx.x + h];
            s[1][threadIdx.x] += s[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(&out[0], s[0][0]);
        atomicAdd(&out[1], s[1][0]);
    }
}

}  // namespace

double relative_residual(const Tree& t, OpsDev& d, const double* f, const double* x, double* tmp, double* scal, cudaStream_t s)
{
    const long N = t.N;
    apply_matvec(t, d, 1, x, tmp, DAFMM_FP64, s);
    UCK(cudaMemsetAsync(scal, 0, 2 * sizeof(double), s));
    resid_kernel<<<(unsigned)std::min<long>(1024, blocks(N)), 256, 0, s>>>(N, (const double2*)f, (const double2*)tmp, scal);
    UCK(cudaGetLastError());
    double h[2];
    UCK(cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, s));
    UCK(cudaStreamSynchronize(s));
    return h[1] > 0 ? std::sqrt(h[0] / h[1]) : 0.0;
}

double* unet_scalars(dafmm_unet* u) { return u->scal + 2; }

}  // namespace dafmm
