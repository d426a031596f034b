// Device-side operator handle shared by the apply kernels and the C-ABI.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

struct dafmm_tree {
    dafmm::Tree t;
};

namespace dafmm {

struct LevelDev {
    int Ri = 0, Ro = 0;
    BsrDev up, m2l, down;
    // coefficient scratch, grown with nrhs: multipoles [slot][Ro][nrhs], locals [slot][Ri][nrhs]
    void* mp64 = nullptr;
    void* lc64 = nullptr;
    void* mp32 = nullptr;
    void* lc32 = nullptr;
};

struct OpsDev {
    std::vector<LevelDev> lv;
    double2* near64 = nullptr;  // 9 x 16 x 16, source offset (sx,sy) -> (sy+1)*3+(sx+1)
    float2* near32 = nullptr;
    int* nbr = nullptr;         // [nleaf][9] source leaf of each near offset, -1 outside
    double* q = nullptr;        // contrast at the N nodes
    float2* v32 = nullptr;      // complex64 copy of the input (mixed precision)
    int nrhs_cap = 0;           // scratch sized for this many right-hand sides
    // per-pass timing: 5 events per profiled call (start, up, m2l, down, leaf)
    bool profile = false;
    std::vector<cudaEvent_t> events;
    size_t ev_used = 0;
};

// Allocate and upload; frees host block storage as it goes.
void upload_ops(const Tree& t, OpsHost& h, OpsDev& d);
void free_ops(OpsDev& d);
void profile_enable(OpsDev& d, bool on);
void profile_read(OpsDev& d, dafmm_profile_t& p);
// Make sure scratch holds nrhs right-hand sides.
void ensure_scratch(const Tree& t, OpsDev& d, int nrhs);
// out = v + kappa^2 q (K~ v), asynchronous on stream.
void apply_matvec(const Tree& t, OpsDev& d, int nrhs, const double* v, double* out, int precision, cudaStream_t stream);
// Same operator, one right-hand side, scratch in a static device array.
void apply_matvec_noalloc(const Tree& t, const OpsDev& d, const double* v, double* out, int precision, cudaStream_t stream);

}  // namespace dafmm

struct dafmm_ops {
    const dafmm_tree* tree = nullptr;
    dafmm::OpsDev dev;
    dafmm::EntryTable table;  // host copy of the offset table (dafmm_entries)
    dafmm_stats_t stats{};
};
