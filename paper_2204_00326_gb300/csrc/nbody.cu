// Direct summation of the point N-body potential of Experiment 1 (Section
// 6.2): u_i = sum_{j != i} G(x_i, x_j) v_j, G = (i/4) H0^(1)(kappa |x - y|),
// over the tree's nodes.  O(N^2): the reference the DAFMM is checked and
// timed against in that experiment.  One warp per target; every lane walks a
// strided share of the sources with the Hankel function evaluated in
// registers (J0 and Y0 in FP64), and the lanes' partial sums are combined by
// warp shuffles in a fixed order.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "ops.h"

namespace dafmm {
namespace {

constexpr int kNbThreads = 256;

__global__ void __launch_bounds__(kNbThreads) nbody_direct_kernel(long N, double kappa, const double2* __restrict__ xy,
                                                                  const double2* __restrict__ v, double2* __restrict__ out)
{
    const long i = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= N) return;  // uniform over the warp
    const double2 pi = xy[i];
    double ar = 0.0, ai = 0.0;
    for (long j = lane; j < N; j += 32) {
        if (j == i) continue;
        const double2 pj = xy[j];
        const double z = kappa * hypot(pi.x - pj.x, pi.y - pj.y);
        const double gr = -0.25 * y0(z), gi = 0.25 * j0(z);
        const double2 vj = __ldg(&v[j]);
        ar += gr * vj.x - gi * vj.y;
        ai += gr * vj.y + gi * vj.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, o);
        ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) out[i] = make_double2(ar, ai);
}

void ck(cudaError_t e, const char* what)
{
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(DAFMM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

}  // namespace

void node_coords(const Tree& t, double* xy)
{
    double z[16];
    cheb_nodes(t.p, z);
    const int n2 = t.p * t.p;
    for (long i = 0; i < t.N; i++) {
        const long leaf = i / n2;
        const int ip = (int)(i % n2);
        const double ax = t.x0 + (2.0 * t.leaf_x[leaf] + 1.0) * t.beta;
        const double ay = t.x0 + (2.0 * t.leaf_y[leaf] + 1.0) * t.beta;
        xy[2 * i] = ax + t.beta * z[ip % t.p];
        xy[2 * i + 1] = ay + t.beta * z[ip / t.p];
    }
}

void node_coords_dev(const Tree& t, double* xy_dev, cudaStream_t s)
{
    std::vector<double> h((size_t)2 * t.N);
    node_coords(t, h.data());
    ck(cudaMemcpyAsync(xy_dev, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, s), "copy of the node coordinates");
    ck(cudaStreamSynchronize(s), "cudaStreamSynchronize");
}

void nbody_direct(const Tree& t, const double* v, double* out, cudaStream_t s)
{
    cudaGetLastError();
    double2* xy = nullptr;
    if (cudaMallocAsync((void**)&xy, sizeof(double2) * (size_t)t.N, s) != cudaSuccess) {
        cudaGetLastError();
        fail(DAFMM_ENOMEM, "device allocation of the node coordinates failed");
    }
    try {
        node_coords_dev(t, (double*)xy, s);
    } catch (...) {
        cudaFreeAsync(xy, s);
        throw;
    }
    const long warps = t.N;
    const unsigned blocks = (unsigned)((warps * 32 + kNbThreads - 1) / kNbThreads);
    nbody_direct_kernel<<<blocks, kNbThreads, 0, s>>>(t.N, t.prm.kappa, xy, (const double2*)v, (double2*)out);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(xy, s);
    ck(e, "nbody_direct_kernel launch");
}

}  // namespace dafmm
