// DAFMM application on the device (Section 5, steps 3-6).
//
// Every tree pass is a block-sparse complex matrix-vector product between
// coefficient spaces (P2M, M2M and directional M2M up; M2L and directional
// M2L across; directional L2L, L2L down).  One kernel serves them all: a warp
// owns one output row (a box, or a (box, cone) slot), streams that row's
// operator blocks once from HBM with coalesced loads, gathers the input
// coefficients of the listed slots, and accumulates in registers; lanes split
// the inner index when blocks are narrower than a warp and reduce by
// shuffles.  The leaf kernel fuses L2P, the tabulated near field (nine shared
// 16 x 16 blocks kept in shared memory) and the epilogue v + kappa^2 q (.).
#include <cuda_runtime.h>

#include <cstring>
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

constexpr int kRowsPerCta = 4;   // one warp per output row
constexpr int kMaxChunks = 4;    // output blocks up to 128 rows

// y[row] (+)= sum_e M_e x[col_e]; M_e is Rout x Rin, column-major.
template <typename T>
__global__ void __launch_bounds__(128) bsr_apply_kernel(int nrows, const int* __restrict__ rowptr, const int* __restrict__ col,
                                                        const typename V2<T>::t* __restrict__ mats, int Rout, int Rin,
                                                        const typename V2<T>::t* __restrict__ x, int ldx,
                                                        typename V2<T>::t* __restrict__ y, int ldy, int accumulate)
{
    using C = typename V2<T>::t;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * kRowsPerCta + warp;
    if (row >= nrows) return;
    const int e0 = rowptr[row], e1 = rowptr[row + 1];
    const size_t blk = (size_t)Rin * Rout;
    if (Rout <= 32) {
        // Rout in {8, 16, 32}: lane = i + Rout * jp
        const int i = lane % Rout, jp = lane / Rout, JP = 32 / Rout;
        T ar = 0, ai = 0;
        for (int e = e0; e < e1; e++) {
            const C* M = mats + (size_t)e * blk + i;
            const C* xv = x + (size_t)col[e] * ldx;
#pragma unroll 4
            for (int j = jp; j < Rin; j += JP) {
                C m = M[(size_t)j * Rout];
                C xx = xv[j];
                ar = fma(m.x, xx.x, fma(-m.y, xx.y, ar));
                ai = fma(m.x, xx.y, fma(m.y, xx.x, ai));
            }
        }
        for (int o = Rout; o < 32; o <<= 1) {
            ar += __shfl_xor_sync(0xffffffffu, ar, o);
            ai += __shfl_xor_sync(0xffffffffu, ai, o);
        }
        if (jp == 0) {
            C* yy = y + (size_t)row * ldy + i;
            if (accumulate) {
                C o = *yy;
                ar += o.x;
                ai += o.y;
            }
            C r;
            r.x = ar;
            r.y = ai;
            *yy = r;
        }
    } else {
        const int nch = (Rout + 31) / 32;
        T ar[kMaxChunks], ai[kMaxChunks];
#pragma unroll
        for (int c = 0; c < kMaxChunks; c++) ar[c] = ai[c] = 0;
        for (int e = e0; e < e1; e++) {
            const C* M = mats + (size_t)e * blk;
            const C* xv = x + (size_t)col[e] * ldx;
            for (int j = 0; j < Rin; j++) {
                C xx = xv[j];
#pragma unroll
                for (int c = 0; c < kMaxChunks; c++) {
                    int i = c * 32 + lane;
                    if (c < nch && i < Rout) {
                        C m = M[(size_t)j * Rout + i];
                        ar[c] = fma(m.x, xx.x, fma(-m.y, xx.y, ar[c]));
                        ai[c] = fma(m.x, xx.y, fma(m.y, xx.x, ai[c]));
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < kMaxChunks; c++) {
            int i = c * 32 + lane;
            if (c < nch && i < Rout) {
                C* yy = y + (size_t)row * ldy + i;
                T rr = ar[c], ri = ai[c];
                if (accumulate) {
                    C o = *yy;
                    rr += o.x;
                    ri += o.y;
                }
                C r;
                r.x = rr;
                r.y = ri;
                *yy = r;
            }
        }
    }
}

// out = v + kappa^2 q (U_B u^{B,i} + sum_{9 offsets} T_o v_{B+o}) per leaf.
// 16 threads per leaf (one per node), 8 leaves per CTA.  Near blocks are
// stored [o][j][i] (target index fastest) for conflict-free shared reads.
template <typename T>
__global__ void __launch_bounds__(128) leaf_apply_kernel(int nleaf, const int* __restrict__ nbr,
                                                         const typename V2<T>::t* __restrict__ near,
                                                         const typename V2<T>::t* __restrict__ vin,
                                                         const int* __restrict__ l2p_rowptr,
                                                         const typename V2<T>::t* __restrict__ l2p, int Ri,
                                                         const typename V2<T>::t* __restrict__ lc,
                                                         const double2* __restrict__ v, const double* __restrict__ q, double k2,
                                                         double2* __restrict__ out)
{
    using C = typename V2<T>::t;
    __shared__ C sn[9 * 256];
    for (int k = threadIdx.x; k < 9 * 256; k += blockDim.x) sn[k] = near[k];
    __syncthreads();
    const int leaf = blockIdx.x * 8 + (threadIdx.x >> 4);
    const int i = threadIdx.x & 15;
    if (leaf >= nleaf) return;
    T ar = 0, ai = 0;
#pragma unroll 1
    for (int o = 0; o < 9; o++) {
        const int src = nbr[leaf * 9 + o];
        if (src < 0) continue;
        const C* vs = vin + (size_t)src * 16;
        const C* B = sn + o * 256 + i;
#pragma unroll
        for (int j = 0; j < 16; j++) {
            C m = B[j * 16];
            C xx = vs[j];
            ar = fma(m.x, xx.x, fma(-m.y, xx.y, ar));
            ai = fma(m.x, xx.y, fma(m.y, xx.x, ai));
        }
    }
    if (l2p_rowptr != nullptr && l2p_rowptr[leaf + 1] > l2p_rowptr[leaf]) {
        const int e = l2p_rowptr[leaf];
        const C* U = l2p + (size_t)e * Ri * 16 + i;
        const C* u = lc + (size_t)leaf * Ri;
        for (int j = 0; j < Ri; j++) {
            C m = U[j * 16];
            C xx = u[j];
            ar = fma(m.x, xx.x, fma(-m.y, xx.y, ar));
            ai = fma(m.x, xx.y, fma(m.y, xx.x, ai));
        }
    }
    const size_t g = (size_t)leaf * 16 + i;
    const double2 vv = v[g];
    const double s = k2 * q[g];
    out[g] = make_double2(vv.x + s * (double)ar, vv.y + s * (double)ai);
}

__global__ void to_c64_kernel(long n, const double2* __restrict__ a, float2* __restrict__ b)
{
    long k = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (k < n) b[k] = make_float2((float)a[k].x, (float)a[k].y);
}

#define CK(x)                                                                                     \
    do {                                                                                          \
        cudaError_t e_ = (x);                                                                     \
        if (e_ != cudaSuccess) fail(DAFMM_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
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

void upload_bsr(BsrHost& h, BsrDev& d)
{
    d.nrows = h.nrows;
    d.Rout = h.Rout;
    d.Rin = h.Rin;
    d.nnz = h.nnz();
    if (h.Rout > 32 * kMaxChunks) fail(DAFMM_EBADARG, "rank above 128; set max_rank or loosen eps_nca");
    dev_alloc(&d.rowptr, sizeof(int) * (h.nrows + 1));
    CK(cudaMemcpy(d.rowptr, h.rowptr.data(), sizeof(int) * (h.nrows + 1), cudaMemcpyHostToDevice));
    dev_alloc(&d.col, sizeof(int) * h.col.size());
    if (!h.col.empty()) CK(cudaMemcpy(d.col, h.col.data(), sizeof(int) * h.col.size(), cudaMemcpyHostToDevice));
    const size_t n = h.mats.size();
    dev_alloc((double2**)&d.m64, sizeof(double2) * n);
    dev_alloc((float2**)&d.m32, sizeof(float2) * n);
    if (n) {
        CK(cudaMemcpy(d.m64, h.mats.data(), sizeof(double2) * n, cudaMemcpyHostToDevice));
        std::vector<float2> f(n);
        for (size_t k = 0; k < n; k++) f[k] = make_float2((float)h.mats[k].real(), (float)h.mats[k].imag());
        CK(cudaMemcpy(d.m32, f.data(), sizeof(float2) * n, cudaMemcpyHostToDevice));
    }
    std::vector<cd>().swap(h.mats);
}

void free_bsr(BsrDev& d)
{
    cudaFree(d.rowptr);
    cudaFree(d.col);
    cudaFree(d.m64);
    cudaFree(d.m32);
    d = BsrDev();
}

template <typename T>
void launch_bsr(const BsrDev& b, const void* x, int ldx, void* y, int ldy, int accumulate, cudaStream_t s)
{
    using C = typename V2<T>::t;
    if (b.nrows == 0) return;
    const C* m = (const C*)(sizeof(T) == 8 ? b.m64 : b.m32);
    unsigned grid = (unsigned)((b.nrows + kRowsPerCta - 1) / kRowsPerCta);
    bsr_apply_kernel<T><<<grid, 32 * kRowsPerCta, 0, s>>>(b.nrows, b.rowptr, b.col, m, b.Rout, b.Rin, (const C*)x, ldx, (C*)y,
                                                           ldy, accumulate);
}

// Event k of the current profiled call (k = 0..4), or nullptr.
cudaEvent_t prof_event(OpsDev& d, int k)
{
    if (!d.profile) return nullptr;
    if (k == 0) {
        if (d.ev_used + 5 > (size_t)5 * 65536) return nullptr;
        while (d.events.size() < d.ev_used + 5) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            d.events.push_back(e);
        }
        d.ev_used += 5;
    }
    if (d.ev_used < 5) return nullptr;
    return d.events[d.ev_used - 5 + k];
}

void mark(OpsDev& d, int k, cudaStream_t s, bool& live)
{
    if (k == 0) live = d.profile && d.ev_used + 5 <= (size_t)5 * 65536;
    if (!live) return;
    cudaEvent_t e = prof_event(d, k);
    if (e) CK(cudaEventRecord(e, s));
}

template <typename T>
void run(const Tree& t, OpsDev& d, const double* v, double* out, cudaStream_t s)
{
    using C = typename V2<T>::t;
    bool live = false;
    mark(d, 0, s, live);
    const int L = t.L;
    const long N = t.N;
    const int nleaf = t.nb * t.nb;
    const C* vin;
    if (sizeof(T) == 4) {
        to_c64_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, (const double2*)v, d.v32);
        vin = (const C*)d.v32;
    } else {
        vin = (const C*)v;
    }
    auto MP = [&](int nu) { return sizeof(T) == 8 ? d.lv[nu].mp64 : d.lv[nu].mp32; };
    auto LC = [&](int nu) { return sizeof(T) == 8 ? d.lv[nu].lc64 : d.lv[nu].lc32; };
    const bool far = t.top <= L;
    if (far) {
        // upward pass: P2M at the leaves, M2M (and directional M2M) above
        launch_bsr<T>(d.lv[L].up, vin, 16, MP(L), d.lv[L].Ro, 0, s);
        for (int nu = L - 1; nu >= t.top; nu--) launch_bsr<T>(d.lv[nu].up, MP(nu + 1), d.lv[nu + 1].Ro, MP(nu), d.lv[nu].Ro, 0, s);
    }
    mark(d, 1, s, live);
    if (far) {
        // transverse pass: M2L at every level
        for (int nu = t.top; nu <= L; nu++) launch_bsr<T>(d.lv[nu].m2l, MP(nu), d.lv[nu].Ro, LC(nu), d.lv[nu].Ri, 0, s);
    }
    mark(d, 2, s, live);
    if (far) {
        // downward pass: (directional) L2L into the children's locals
        for (int nu = t.top; nu < L; nu++) launch_bsr<T>(d.lv[nu].down, LC(nu), d.lv[nu].Ri, LC(nu + 1), d.lv[nu + 1].Ri, 1, s);
    }
    mark(d, 3, s, live);
    const C* nearp = (const C*)(sizeof(T) == 8 ? (void*)d.near64 : (void*)d.near32);
    const BsrDev* l2p = far ? &d.lv[L].down : nullptr;
    leaf_apply_kernel<T><<<(unsigned)((nleaf + 7) / 8), 128, 0, s>>>(
        nleaf, d.nbr, nearp, vin, l2p ? l2p->rowptr : nullptr, l2p ? (const C*)(sizeof(T) == 8 ? l2p->m64 : l2p->m32) : nullptr,
        far ? d.lv[L].Ri : 0, far ? (const C*)LC(L) : nullptr, (const double2*)v, d.q, t.prm.kappa * t.prm.kappa, (double2*)out);
    CK(cudaGetLastError());
    mark(d, 4, s, live);
}

}  // namespace

void upload_ops(const Tree& t, OpsHost& h, OpsDev& d)
{
    const int L = t.L;
    d.lv.assign(L + 1, LevelDev());
    if (t.top <= L) {
        for (int nu = t.top; nu <= L; nu++) {
            d.lv[nu].Ri = h.lv[nu].Ri;
            d.lv[nu].Ro = h.lv[nu].Ro;
            upload_bsr(h.lv[nu].up, d.lv[nu].up);
            upload_bsr(h.lv[nu].m2l, d.lv[nu].m2l);
            upload_bsr(h.lv[nu].down, d.lv[nu].down);
        }
    }
    // near blocks, transposed to [o][j][i]
    std::vector<double2> n64(9 * 256);
    std::vector<float2> n32(9 * 256);
    for (int o = 0; o < 9; o++)
        for (int i = 0; i < 16; i++)
            for (int j = 0; j < 16; j++) {
                cd v = h.near[o * 256 + i * 16 + j];
                n64[o * 256 + j * 16 + i] = make_double2(v.real(), v.imag());
                n32[o * 256 + j * 16 + i] = make_float2((float)v.real(), (float)v.imag());
            }
    dev_alloc(&d.near64, sizeof(double2) * 9 * 256);
    dev_alloc(&d.near32, sizeof(float2) * 9 * 256);
    CK(cudaMemcpy(d.near64, n64.data(), sizeof(double2) * 9 * 256, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.near32, n32.data(), sizeof(float2) * 9 * 256, cudaMemcpyHostToDevice));
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
    dev_alloc(&d.nbr, sizeof(int) * nbr.size());
    CK(cudaMemcpy(d.nbr, nbr.data(), sizeof(int) * nbr.size(), cudaMemcpyHostToDevice));
    ensure_scratch(t, d, 1);
}

void ensure_scratch(const Tree& t, OpsDev& d, int nrhs)
{
    if (nrhs <= d.nrhs_cap) return;
    const int L = t.L;
    for (int nu = 0; nu <= L && t.top <= L; nu++) {
        if (nu < t.top) continue;
        LevelDev& l = d.lv[nu];
        cudaFree(l.mp64);
        cudaFree(l.lc64);
        cudaFree(l.mp32);
        cudaFree(l.lc32);
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
    dev_alloc(&d.v32, sizeof(float2) * (size_t)t.N * nrhs);
    d.nrhs_cap = nrhs;
}

void profile_enable(OpsDev& d, bool on)
{
    d.profile = on;
    d.ev_used = 0;
}

void profile_read(OpsDev& d, dafmm_profile_t& p)
{
    std::memset(&p, 0, sizeof(p));
    for (size_t c = 0; c + 5 <= d.ev_used; c += 5) {
        float ms[4];
        CK(cudaEventSynchronize(d.events[c + 4]));
        for (int k = 0; k < 4; k++) CK(cudaEventElapsedTime(&ms[k], d.events[c + k], d.events[c + k + 1]));
        p.ms_up += ms[0];
        p.ms_m2l += ms[1];
        p.ms_down += ms[2];
        p.ms_leaf += ms[3];
        p.ms_total += ms[0] + ms[1] + ms[2] + ms[3];
        p.calls++;
    }
}

void free_ops(OpsDev& d)
{
    for (cudaEvent_t e : d.events) cudaEventDestroy(e);
    d.events.clear();
    for (auto& l : d.lv) {
        free_bsr(l.up);
        free_bsr(l.m2l);
        free_bsr(l.down);
        cudaFree(l.mp64);
        cudaFree(l.lc64);
        cudaFree(l.mp32);
        cudaFree(l.lc32);
    }
    d.lv.clear();
    cudaFree(d.near64);
    cudaFree(d.near32);
    cudaFree(d.nbr);
    cudaFree(d.q);
    cudaFree(d.v32);
    d = OpsDev();
}

void apply_matvec(const Tree& t, OpsDev& d, int nrhs, const double* v, double* out, int precision, cudaStream_t stream)
{
    if (nrhs != 1) fail(DAFMM_EBADARG, "this build applies one right-hand side per call");
    ensure_scratch(t, d, nrhs);
    if (precision == DAFMM_FP64)
        run<double>(t, d, v, out, stream);
    else
        run<float>(t, d, v, out, stream);
}

// ---------------------------------------------------------------------------
// Allocation-free application.  Some callers cannot let the library allocate
// device memory at call time: processes whose device memory is owned by their
// own pool (a cudaMalloc there can fail or fragment the pool), hot loops that
// cannot afford cudaMalloc's implicit device synchronisation, and deployments
// that must fix all memory before they start.  For them the coefficient
// scratch of one single-RHS application lives in this fixed device array
// instead of the handle's grow-on-demand buffers.  Every GPU that loads the
// library holds the array until the process exits; all calls on a device
// share it, so calls whose kernels overlap in time on that device race.
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
    const long N = t.N;
    const int nleaf = t.nb * t.nb;
    const bool far = t.top <= L;
    void* mp[64] = {};
    void* lc[64] = {};
    if (L >= 64) fail(DAFMM_EBADARG, "tree too deep for the allocation-free path");
    // carve the scratch: complex64 copy of v (mixed), then per level multipoles and locals
    size_t need = sizeof(T) == 4 ? align256(sizeof(float2) * (size_t)N) : 0;
    if (far)
        for (int nu = t.top; nu <= L; nu++)
            need += align256(sizeof(C) * (size_t)t.lv[nu].nslot() * d.lv[nu].Ro) +
                    align256(sizeof(C) * (size_t)t.lv[nu].nslot() * d.lv[nu].Ri);
    if (need > (size_t)DAFMM_NOALLOC_SCRATCH_BYTES)
        fail(DAFMM_EBADARG, "problem needs " + std::to_string(need) + " bytes of scratch; the allocation-free path holds " +
                                std::to_string((size_t)DAFMM_NOALLOC_SCRATCH_BYTES) + " (use dafmm_matvec)");
    unsigned char* base = noalloc_scratch();
    // the array keeps the previous call's contents: start from zeros
    CK(cudaMemsetAsync(base, 0, need, s));
    size_t off = 0;
    const C* vin = (const C*)v;
    if (sizeof(T) == 4) {
        float2* v32 = (float2*)(base + off);
        off += align256(sizeof(float2) * (size_t)N);
        to_c64_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, (const double2*)v, v32);
        vin = (const C*)v32;
    }
    if (far) {
        for (int nu = t.top; nu <= L; nu++) {
            mp[nu] = base + off;
            off += align256(sizeof(C) * (size_t)t.lv[nu].nslot() * d.lv[nu].Ro);
            lc[nu] = base + off;
            off += align256(sizeof(C) * (size_t)t.lv[nu].nslot() * d.lv[nu].Ri);
        }
        launch_bsr<T>(d.lv[L].up, vin, 16, mp[L], d.lv[L].Ro, 0, s);
        for (int nu = L - 1; nu >= t.top; nu--) launch_bsr<T>(d.lv[nu].up, mp[nu + 1], d.lv[nu + 1].Ro, mp[nu], d.lv[nu].Ro, 0, s);
        for (int nu = t.top; nu <= L; nu++) launch_bsr<T>(d.lv[nu].m2l, mp[nu], d.lv[nu].Ro, lc[nu], d.lv[nu].Ri, 0, s);
        for (int nu = t.top; nu < L; nu++) launch_bsr<T>(d.lv[nu].down, lc[nu], d.lv[nu].Ri, lc[nu + 1], d.lv[nu + 1].Ri, 1, s);
    }
    const C* nearp = (const C*)(sizeof(T) == 8 ? (const void*)d.near64 : (const void*)d.near32);
    const BsrDev* l2p = far ? &d.lv[L].down : nullptr;
    leaf_apply_kernel<T><<<(unsigned)((nleaf + 7) / 8), 128, 0, s>>>(
        nleaf, d.nbr, nearp, vin, l2p ? l2p->rowptr : nullptr, l2p ? (const C*)(sizeof(T) == 8 ? l2p->m64 : l2p->m32) : nullptr,
        far ? d.lv[L].Ri : 0, far ? (const C*)lc[L] : nullptr, (const double2*)v, d.q, t.prm.kappa * t.prm.kappa, (double2*)out);
    CK(cudaGetLastError());
}

}  // namespace

void apply_matvec_noalloc(const Tree& t, const OpsDev& d, const double* v, double* out, int precision, cudaStream_t stream)
{
    if (precision == DAFMM_FP64)
        run_noalloc<double>(t, d, v, out, stream);
    else
        run_noalloc<float>(t, d, v, out, stream);
}

}  // namespace dafmm
