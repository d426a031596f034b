// Several problems of different sizes in one application, and the tuner of
// the several-right-hand-side passes.
//
// dafmm_batch: the problems' operator applications are captured once (per
// right-hand-side count, precision and set of vector pointers) into one CUDA
// graph: with several right-hand sides every problem on its own stream forked
// from and joined to the capture stream, so small problems' kernels run
// beside large ones' (their kernels never wait on other CTAs); with one
// right-hand side in order (the fused kernel's warps wait on each other, so
// two of them must not share the GPU); each call replays the graph with one
// cudaGraphLaunch.
//
// dafmm_tune_batched: times the candidate configurations of an operator's
// several-right-hand-side passes with CUDA events and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ops.h"

struct dafmm_batch {
    std::vector<dafmm_ops*> ops;
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> lanes;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    struct Entry {
        int nrhs = 0, precision = 0;
        std::vector<const double*> v;
        std::vector<double*> out;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        unsigned long long used = 0;
    };
    std::vector<Entry> cache;  // at most kBatchGraphs captured applications
    unsigned long long clock = 0;
};

namespace dafmm {
namespace {

constexpr size_t kBatchGraphs = 4;

void ck(cudaError_t e, const char* what)
{
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(DAFMM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

void drop(dafmm_batch::Entry& e)
{
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.graph) cudaGraphDestroy(e.graph);
    e.exec = nullptr;
    e.graph = nullptr;
}

}  // namespace

dafmm_batch* batch_new(int n, dafmm_ops* const* ops)
{
    dafmm_batch* b = new dafmm_batch();
    try {
        b->ops.assign(ops, ops + n);
        ck(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "cudaStreamCreate");
        ck(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "cudaEventCreate");
        b->lanes.assign(n, nullptr);
        b->join.assign(n, nullptr);
        for (int i = 0; i < n; i++) {
            ck(cudaStreamCreateWithFlags(&b->lanes[i], cudaStreamNonBlocking), "cudaStreamCreate");
            ck(cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming), "cudaEventCreate");
        }
    } catch (...) {
        batch_free(b);
        throw;
    }
    return b;
}

size_t batch_size(const dafmm_batch* b) { return b->ops.size(); }

void batch_free(dafmm_batch* b)
{
    if (!b) return;
    for (auto& e : b->cache) drop(e);
    for (cudaStream_t s : b->lanes)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

void batch_matvec(dafmm_batch* b, int nrhs, const double* const* v, double* const* out, int precision, cudaStream_t s)
{
    const int n = (int)b->ops.size();
    dafmm_batch::Entry* hit = nullptr;
    for (auto& e : b->cache)
        if (e.exec && e.nrhs == nrhs && e.precision == precision && std::equal(e.v.begin(), e.v.end(), v) &&
            std::equal(e.out.begin(), e.out.end(), out))
            hit = &e;
    if (!hit) {
        // scratch first: nothing may allocate inside the capture
        for (int i = 0; i < n; i++) ensure_scratch(b->ops[i]->tree->t, b->ops[i]->dev, nrhs);
        if (b->cache.size() < kBatchGraphs) b->cache.emplace_back();
        dafmm_batch::Entry* e = &b->cache[0];
        for (auto& c : b->cache)
            if (!c.exec || c.used < e->used) e = &c;
        drop(*e);
        cudaGraph_t g = nullptr;
        ck(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        try {
            if (nrhs == 1) {
                // one right-hand side runs the cooperative fused kernel, whose warps wait on
                // each other: two of them must not share the GPU, so the problems run in order
                for (int i = 0; i < n; i++) apply_matvec(b->ops[i]->tree->t, b->ops[i]->dev, 1, v[i], out[i], precision, b->cap);
            } else {
                ck(cudaEventRecord(b->fork, b->cap), "cudaEventRecord");
                for (int i = 0; i < n; i++) {
                    ck(cudaStreamWaitEvent(b->lanes[i], b->fork, 0), "cudaStreamWaitEvent");
                    apply_matvec(b->ops[i]->tree->t, b->ops[i]->dev, nrhs, v[i], out[i], precision, b->lanes[i]);
                    ck(cudaEventRecord(b->join[i], b->lanes[i]), "cudaEventRecord");
                    ck(cudaStreamWaitEvent(b->cap, b->join[i], 0), "cudaStreamWaitEvent");
                }
            }
        } catch (...) {
            cudaStreamEndCapture(b->cap, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            throw;
        }
        ck(cudaStreamEndCapture(b->cap, &g), "cudaStreamEndCapture");
        e->graph = g;
        ck(cudaGraphInstantiate(&e->exec, g, 0), "cudaGraphInstantiate");
        e->nrhs = nrhs;
        e->precision = precision;
        e->v.assign(v, v + n);
        e->out.assign(out, out + n);
        hit = e;
    }
    hit->used = ++b->clock;
    ck(cudaGraphLaunch(hit->exec, s), "cudaGraphLaunch");
}

namespace {
__global__ void fill_kernel(long n, double2* x)
{
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < n) {
        // a deterministic pseudo-random pattern (Weyl sequence), values in [-1, 1]
        const double a = (double)((i * 2654435761ul) & 0xffff) / 32768.0 - 1.0;
        const double c = (double)((i * 40503ul + 12345ul) & 0xffff) / 32768.0 - 1.0;
        x[i] = make_double2(a, c);
    }
}
}  // namespace

void tune_batched(dafmm_ops* ops, int nrhs, int precision, dafmm_tuning& r)
{
    OpsDev& d = ops->dev;
    const Tree& t = ops->tree->t;
    const long n = t.N * (long)nrhs;
    const int keep_kernel = d.batched_kernel, keep_cps = d.batched_cps;
    double2 *v = nullptr, *o = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        cudaFree(v);
        cudaFree(o);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
    };
    try {
        if (cudaMalloc(&v, sizeof(double2) * n) != cudaSuccess || cudaMalloc(&o, sizeof(double2) * n) != cudaSuccess) {
            cudaGetLastError();
            fail(DAFMM_ENOMEM, "device allocation of the tuning vectors failed");
        }
        ck(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "cudaStreamCreate");
        ck(cudaEventCreate(&e0), "cudaEventCreate");
        ck(cudaEventCreate(&e1), "cudaEventCreate");
        fill_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, v);
        ck(cudaGetLastError(), "fill_kernel");
        struct Cand {
            int kernel, cps;
        };
        std::vector<Cand> cands = {{1, 0}, {1, 1}, {1, 2}, {1, 4}};
        if (precision == DAFMM_MIXED) cands.push_back({2, 0});
        r.ncand = 0;
        double best = 1e300;
        for (const Cand& c : cands) {
            set_batched_kernel(d, c.kernel);
            set_batched_grid(d, c.cps);
            for (int k = 0; k < 2; k++) apply_matvec(t, d, nrhs, (const double*)v, (double*)o, precision, s);
            ck(cudaEventRecord(e0, s), "cudaEventRecord");
            constexpr int reps = 5;
            for (int k = 0; k < reps; k++) apply_matvec(t, d, nrhs, (const double*)v, (double*)o, precision, s);
            ck(cudaEventRecord(e1, s), "cudaEventRecord");
            ck(cudaEventSynchronize(e1), "cudaEventSynchronize");
            float ms = 0;
            ck(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
            const double per = ms / reps;
            r.cand_kernel[r.ncand] = c.kernel;
            r.cand_ctas[r.ncand] = c.cps;
            r.cand_ms[r.ncand] = per;
            r.ncand++;
            if (per < best) {
                best = per;
                r.kernel = c.kernel;
                r.ctas_per_sm = c.cps;
            }
        }
        r.nrhs = nrhs;
        r.precision = precision;
        r.best_ms = best;
        set_batched_kernel(d, r.kernel);
        set_batched_grid(d, r.ctas_per_sm);
    } catch (...) {
        set_batched_kernel(d, keep_kernel);
        set_batched_grid(d, keep_cps);
        cleanup();
        throw;
    }
    cleanup();
}

}  // namespace dafmm
