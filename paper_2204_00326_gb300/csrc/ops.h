// Device-side operator handle shared by the apply kernels and the C-ABI.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

struct dafmm_tree {
    dafmm::Tree t;
};

namespace dafmm {

// Operators of one level and its coefficient scratch.
struct LevelDev {
    int Ri = 0, Ro = 0;  // strides of the local / multipole buffers
    BsrDev up, m2l, down;
    BsrDev upc;  // level L-1 only: its up pass composed with the leaves' P2M (reads the input vector)
    // coefficient scratch, grown with nrhs: multipoles [slot][Ro][nrhs], locals [slot][Ri][nrhs]
    void* mp64 = nullptr;
    void* lc64 = nullptr;
    void* mp32 = nullptr;
    void* lc32 = nullptr;
    // single right-hand side, [0] complex128, [1] complex64: multipoles, locals
    // from M2L, locals from the parent (L2L); rows no pass writes stay zero
    void* fmp[2] = {};
    void* flc[2] = {};
    void* flcd[2] = {};
};

// Block-sparse passes launched together: their rows are cut into chunks of
// at most a thousand block entries; chunk ranges go to warps (one right-hand
// side) or CTAs (several), and the last writer of a split row sums its
// partials in a fixed order.
struct PassRef {
    int level = 0;
    int kind = 0;  // 0 up (P2M/M2M), 1 M2L, 2 down (L2L), 3 up of level L-1 composed with P2M
};

struct Group {
    std::vector<PassRef> passes;
    int nch = 0;             // chunks
    int Pld = 0;             // stride of a chunk's partial (largest row rank)
    int4* chunks = nullptr;  // two int4 per chunk (a column range of a row's matrix), see apply.cu
    int accumulate = 0;      // add into y instead of overwriting
    int* cnt = nullptr;      // per chunk: writers of a split row's partials seen so far
    // per pass: element offset of each row's matrix, offset of each row's
    // columns in xmap, and for every column the index of its input coefficient
    std::vector<long*> rbase;
    std::vector<int*> cbase;
    std::vector<int*> xmap;
    std::vector<int> xmap_n;  // per pass: columns in xmap
};

// Every tree pass of a single-right-hand-side application in one cooperative
// launch.  The passes on the dependent chain are ordered by phase and every
// warp takes a fixed share of each phase.  The passes with slack either sit
// in the phases too (complex64: bandwidth-bound, they stream in one long
// phase) or are cut into pieces that warps take from a counter while the
// chain waits (complex128: arithmetic-bound, they fill the chain's latency).
// Before the first chunk of a pass a warp waits until the passes it reads
// have written all their rows (per-pass row counters).
struct FusedPlan {
    int4* chunks = nullptr;        // the chain list (phase by phase), then the bulk list
    int* cnt = nullptr;            // per chunk: counter of a split row starting there
    int nch = 0;
    int nph = 0;
    std::vector<int> base;         // per chain phase: first chunk; base[nph] = chain chunks
    std::vector<unsigned> phdeps;  // per chain phase: passes read by its passes
    std::vector<int> wlo, wn;      // per chain phase: the warps sharing it (empty: every warp)
    bool chain_split = false;      // the chain phases after the first have warps of their own (which take no pieces)
    int npieces = 0;               // bulk pieces (chunk ranges of one row), taken in order
    int4* pieces = nullptr;        // per piece: {first chunk, end chunk, partial slot, pass}
    size_t part = 0;               // complex elements of chunk partials it uses
};

struct Fused {
    Group g;                       // passes and their tables (g.chunks unused)
    std::vector<unsigned> deps;    // per pass: bit mask of the passes whose output it reads
    std::vector<int> target;       // per pass: rows it writes
    std::vector<int> dphase;       // per pass: latest phase among the passes it reads (-1: none)
    FusedPlan plan[2];             // [0] complex128, [1] complex64
    int ctas[2] = {0, 0};          // persistent grid, [0] complex128, [1] complex64
    int* done = nullptr;           // per pass: rows written in the running application; then the piece counter
    double cmacs = 0;              // complex multiply-adds of one launch (realised ranks)
    double leaf_cmacs = 0;         // ... of the leaf kernel after it (near field, L2P, composed L2L)
    int leaf_fcc = 0, leaf_fcl = 0;  // leaf kernel: composed and L2P columns staged a leaf (0, 0: not staged)
    int leaf_fcc_plan = 0, leaf_fcl_plan = 0;  // ... as planned (the staging can be switched off)
};

// One captured application (per precision), replayed while the vector
// pointers stay the same.
struct GraphCache {
    cudaGraph_t graph = nullptr;      // the graph exec was instantiated from (owns ev_node)
    cudaGraphExec_t exec = nullptr;
    const double* v = nullptr;
    double* out = nullptr;
    int nrhs = 0;
    cudaGraphNode_t ev_node[5] = {};  // event-record nodes of the five pass marks
    bool marks = false;               // captured with the pass marks (profiled calls)
    unsigned long long used = 0;      // last use (LRU replacement)
};
constexpr int kGraphSlots = 4;        // cached (v, out) pairs per precision

struct GmresWork;  // GMRES workspace kept between solves (gmres.cu)
void gmres_work_free(GmresWork* w);
struct GmresMany;  // the same for several right-hand sides
void gmres_many_free(GmresMany* w);

struct OpsDev {
    std::vector<LevelDev> lv;
    std::vector<Group> up;      // per level (index = level)
    Group m2l;                  // every level at once
    std::vector<Group> down;    // per level (index = parent level)
    Fused fz;                   // single right-hand side: every pass in one launch
    BsrDev leafc;               // rows leaves: the L2L from level L-1 composed with L2P (16 x R per block)
    double2* near64 = nullptr;  // 9 x 16 x 16, source offset (sx,sy) -> (sy+1)*3+(sx+1)
    float4* neardf = nullptr;   // the same as float pairs {re hi, im hi, re lo, im lo}
    float2* near32 = nullptr;
    int* nbr = nullptr;         // [nleaf][9] source leaf of each near offset, -1 outside
    double* q = nullptr;        // contrast at the N nodes
    float2* v32 = nullptr;      // complex64 copy of the input (mixed precision)
    float4* vdf = nullptr;      // float-pair copy of the input (several right-hand sides, complex128)
    void* part = nullptr;       // chunk partials of the largest group (complex128 size)
    size_t part_elems = 0;      // complex elements per right-hand side in part
    int nrhs_cap = 0;           // scratch sized for this many right-hand sides
    int* err = nullptr;         // device flag: a bounded wait in a kernel gave up
    int stall_pass = -1;        // test support: the next fused launch waits for a row this pass never writes
    bool potential = false;     // the leaf epilogue writes K v (apply_potential)
    // per-pass timing: 5 events per profiled call (start, up, m2l, down, leaf);
    // for a fused call the first interval holds the whole far field
    bool profile = false;
    std::vector<cudaEvent_t> events;
    std::vector<char> ev_fused;  // per profiled call
    size_t ev_used = 0;
    // graph replay
    cudaStream_t cap_stream = nullptr;   // private stream used only for capture
    cudaEvent_t placeholder[5] = {};     // events recorded by freshly captured graphs
    GraphCache gc[2][kGraphSlots];
    unsigned long long gc_clock = 0;
    GmresWork* gw = nullptr;
    GmresMany* gm = nullptr;
    int batched_kernel = 0;     // several right-hand sides, complex64: 0 automatic, 1 CUDA cores, 2 tensor cores
    int batched_cps = 0;        // several right-hand sides, CUDA cores: CTAs per SM of the pass grids (0: as many as fit)
};

// Allocate and upload; frees host block storage as it goes.
void upload_ops(const Tree& t, OpsHost& h, OpsDev& d);
void free_ops(OpsDev& d);
void profile_enable(OpsDev& d, bool on);
void set_batched_kernel(OpsDev& d, int mode);
void set_batched_grid(OpsDev& d, int ctas_per_sm);
void set_leaf_staging(OpsDev& d, bool on);
void profile_read(OpsDev& d, dafmm_profile_t& p);
// Make sure scratch holds nrhs right-hand sides.
void ensure_scratch(const Tree& t, OpsDev& d, int nrhs);
// out = v + kappa^2 q (K~ v), asynchronous on stream.
void apply_matvec(const Tree& t, OpsDev& d, int nrhs, const double* v, double* out, int precision, cudaStream_t stream);
// out = K~ v (the volume potential at the nodes, no identity and no kappa^2 q), same kernels.
void apply_potential(const Tree& t, OpsDev& d, int nrhs, const double* v, double* out, int precision, cudaStream_t stream);
// Same operator, one right-hand side, scratch in a static device array.
void apply_matvec_noalloc(const Tree& t, const OpsDev& d, const double* v, double* out, int precision, cudaStream_t stream);
// GMRES (gmres.cu); prec: z = M^{-1} v, or nullptr.
using PrecFn = void (*)(const void* M, const double* v, double* z, int precision, cudaStream_t s);
int gmres_run(const Tree& t, OpsDev& d, const void* M, PrecFn prec, const double* f, double* x, const gmres_opts& o, gmres_stats& st,
              cudaStream_t s);
// nrhs in 2..64 columns [N][nrhs] in lockstep; prec: z = M^{-1} v for all columns, or nullptr; st: nrhs entries
using PrecManyFn = void (*)(const void* M, int nrhs, const double* v, double* z, int precision, cudaStream_t s);
int gmres_run_many(const Tree& t, OpsDev& d, const void* M, PrecManyFn prec, int nrhs, const double* f, double* x, const gmres_opts& o,
                   gmres_stats* st, cudaStream_t s);

// HODLR (hodlr.cu)
dafmm_hodlr* hodlr_build(const dafmm_ops* ops, int rank, double tol, int leaf);
void hodlr_free(dafmm_hodlr* h);
void hodlr_apply(const dafmm_hodlr* h, const double* b, double* x, int precision, cudaStream_t s);
void hodlr_prec(const void* M, const double* v, double* z, int precision, cudaStream_t s);
// nrhs in 2..64 columns stored [N][nrhs]: per-level launches, no device waits
void hodlr_apply_many(const dafmm_hodlr* h, int nrhs, const double* b, double* x, int precision, cudaStream_t s);
void hodlr_prec_many(const void* M, int nrhs, const double* v, double* z, int precision, cudaStream_t s);
// Synchronise s; DAFMM_ETIMEOUT (flag cleared, counters re-armed) when an apply gave up a wait.
int hodlr_check(const dafmm_hodlr* h, cudaStream_t s);
void hodlr_set_stall(const dafmm_hodlr* h, int on);
void hodlr_set_width(dafmm_hodlr* h, int ctas);
const dafmm_tree* hodlr_tree(const dafmm_hodlr* h);
void hodlr_dense(const dafmm_hodlr* h, cd* out);
void hodlr_shape(const dafmm_hodlr* h, long* N, int* levels, int* leaf, int* rank_max, double* seconds);

// Learned guess (unet.cu)
dafmm_unet* unet_new(const unet_params& p);
void unet_delete(dafmm_unet* u);
long unet_size(const dafmm_unet* u);
void unet_get(const dafmm_unet* u, float* host);
void unet_set(dafmm_unet* u, const float* host);
void unet_get_grad(const dafmm_unet* u, float* host);
void unet_fwd(dafmm_unet* u, int B, int H, int W, const float* in, float* out, cudaStream_t s);
double unet_bwd(dafmm_unet* u, int B, int H, int W, const float* in, const float* target, float* out, cudaStream_t s);
void unet_adam_step(dafmm_unet* u, float lr, float b1, float b2, float eps, cudaStream_t s);
// x = a x + c s N(q, v / s) on the tree's node grid, s = max |v|
void unet_apply_nodes(dafmm_unet* u, const Tree& t, const OpsDev& d, const double* v, double* x, double a, double c, cudaStream_t s);

// |f - A x| / |f| with the FP64 operator; tmp: N complex128, scal: 2 device doubles
double relative_residual(const Tree& t, OpsDev& d, const double* f, const double* x, double* tmp, double* scal, cudaStream_t s);
double* unet_scalars(dafmm_unet* u);  // 2 device doubles owned by the network

// Node coordinates (N x 2, the documented order) on the host or, synchronising
// s, copied to the device; the direct N-body sum of Experiment 1 (nbody.cu).
void node_coords(const Tree& t, double* xy);
void node_coords_dev(const Tree& t, double* xy_dev, cudaStream_t s);
void nbody_direct(const Tree& t, const double* v, double* out, cudaStream_t s);
// psi(x_k) (Eq. 7) and u(x_k) = V[psi](x_k) at m points (entries.cu)
void field_eval(const Tree& t, const double* psi, long m, const double* pts, double* u, double* psi_at, cudaStream_t s);

// Several problems in one captured application; the tuner (batch.cpp).
dafmm_batch* batch_new(int n, dafmm_ops* const* ops);
void batch_free(dafmm_batch* b);
size_t batch_size(const dafmm_batch* b);
void batch_matvec(dafmm_batch* b, int nrhs, const double* const* v, double* const* out, int precision, cudaStream_t s);
void tune_batched(dafmm_ops* ops, int nrhs, int precision, dafmm_tuning& r);

// Kernels one application launches.
int launches_per_call(const Tree& t, const OpsDev& d, int precision);
// Synchronise the stream and report (and clear) a device-side wait timeout.
int sync_and_check(OpsDev& d, cudaStream_t stream);

}  // namespace dafmm

struct dafmm_ops {
    const dafmm_tree* tree = nullptr;
    dafmm::OpsDev dev;
    dafmm::EntryTable table;  // host copy of the offset table (dafmm_entries)
    dafmm_stats_t stats{};
};
