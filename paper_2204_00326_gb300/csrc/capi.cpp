// C-ABI entry points of the DAFMM library (declared in include/dafmm.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "ops.h"

namespace dafmm {
namespace {
thread_local int g_last_code = DAFMM_OK;
thread_local std::string g_last_msg;
}  // namespace

void set_last_error(int code, const std::string& msg)
{
    g_last_code = code;
    g_last_msg = msg;
}

template <typename F>
int guarded(F&& f)
{
    try {
        f();
        set_last_error(DAFMM_OK, "");
        return DAFMM_OK;
    } catch (const Status& s) {
        set_last_error(s.code, s.what());
        return s.code;
    } catch (const std::bad_alloc&) {
        set_last_error(DAFMM_ENOMEM, "host allocation failed");
        return DAFMM_ENOMEM;
    } catch (const std::exception& e) {
        set_last_error(DAFMM_EBADARG, e.what());
        return DAFMM_EBADARG;
    }
}

void require_device()
{
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        fail(DAFMM_ECUDA, "no CUDA device available");
    }
}

// Realised (unpadded) work of one application, for the roofline figures.
void fill_stats(const Tree& t, const OpsHost& h, dafmm_stats_t& st)
{
    const int L = t.L;
    double bytes_real = 0, cmacs = 0, vec = 0, c_up = 0, c_m2l = 0, c_down = 0, c_leaf = 0;
    for (int nu = 0; nu <= L && nu < 32; nu++) {
        if (nu < t.top) continue;
        const Level& l = t.lv[nu];
        const LevelOpsHost& lo = h.lv[nu];
        long act = 0;
        double si = 0, so = 0;
        int mi = 0, mo = 0;
        for (int s = 0; s < l.nslot(); s++) {
            if (!l.active[s]) continue;
            act++;
            si += lo.ri[s];
            so += lo.ro[s];
            mi = std::max(mi, lo.ri[s]);
            mo = std::max(mo, lo.ro[s]);
        }
        st.slots[nu] = act;
        st.rank_in_max[nu] = mi;
        st.rank_out_max[nu] = mo;
        st.rank_in_mean[nu] = act ? si / act : 0;
        st.rank_out_mean[nu] = act ? so / act : 0;
        vec += 2.0 * 16.0 * (si + so);  // write + read of locals and multipoles
        // M2L
        for (int s = 0; s < l.nslot(); s++) {
            if (!l.active[s]) continue;
            for (int e = l.il_ptr[s]; e < l.il_ptr[s + 1]; e++) c_m2l += (double)lo.ri[s] * lo.ro[l.il_idx[e]];
        }
        // up / down transfers
        std::vector<int> ch;
        for (int s = 0; s < l.nslot(); s++) {
            if (!l.active[s]) continue;
            if (nu == L) {
                c_up += 16.0 * lo.ro[s];
                c_leaf += 16.0 * lo.ri[s];
            } else {
                child_slots(t, nu, s, ch);
                for (int c : ch) {
                    c_up += (double)lo.ro[s] * h.lv[nu + 1].ro[c];
                    c_down += (double)lo.ri[s] * h.lv[nu + 1].ri[c];
                }
            }
        }
    }
    cmacs = c_up + c_m2l + c_down + c_leaf;
    bytes_real = cmacs * 16.0;  // every far-field operator entry is read once per application
    const long nleaf = (long)t.nb * t.nb;
    long p2p = 0;
    for (int b = 0; b < nleaf; b++)
        for (int sy = -1; sy <= 1; sy++)
            for (int sx = -1; sx <= 1; sx++) {
                int x = t.leaf_x[b] + sx, y = t.leaf_y[b] + sy;
                if (x >= 0 && y >= 0 && x < t.nb && y < t.nb) p2p += 256;
            }
    st.p2p_cmacs_per_rhs = p2p;
    st.cmacs_per_rhs = cmacs + (double)p2p;
    st.operator_bytes_fp64 = bytes_real + 9 * 256 * 16.0;
    st.operator_bytes_fp32 = bytes_real / 2 + 9 * 256 * 8.0;
    st.vector_bytes_per_rhs = vec + (double)t.N * (16 + 16 + 8);
    st.cmacs_up = c_up;
    st.cmacs_m2l = c_m2l;
    st.cmacs_down = c_down;
    st.cmacs_leaf = c_leaf + (double)p2p;
    st.coef_bytes_per_rhs = vec;
}

}  // namespace dafmm

using namespace dafmm;

extern "C" {

int dafmm_last_error(char* buf, size_t size)
{
    if (buf && size) {
        std::snprintf(buf, size, "%s", g_last_msg.c_str());
    }
    return g_last_code;
}

int build_tree(const dafmm_params* params, int n_side, double x0, double x1, dafmm_tree** out)
{
    return guarded([&] {
        if (!params || !out) fail(DAFMM_EBADARG, "NULL argument");
        *out = nullptr;
        Tree* t = make_tree(*params, n_side, x0, x1);
        dafmm_tree* h = new dafmm_tree();
        h->t = std::move(*t);
        delete t;
        *out = h;
    });
}

int tree_nodes(const dafmm_tree* tree, double* xy)
{
    return guarded([&] {
        if (!tree || !xy) fail(DAFMM_EBADARG, "NULL argument");
        node_coords(tree->t, xy);
    });
}

int tree_nodes_dev(const dafmm_tree* tree, double* xy_dev, void* stream)
{
    return guarded([&] {
        if (!tree || !xy_dev) fail(DAFMM_EBADARG, "NULL argument");
        require_device();
        node_coords_dev(tree->t, xy_dev, (cudaStream_t)stream);
    });
}

int dafmm_field_eval(const dafmm_ops* ops, const double* psi, long m, const double* pts, double* u, double* psi_at, void* stream)
{
    return guarded([&] {
        if (!ops || !psi || (m > 0 && (!pts || !u))) fail(DAFMM_EBADARG, "NULL argument");
        if (m < 0 || m > 0x7fffffffL) fail(DAFMM_EBADARG, "point count out of range");
        require_device();
        field_eval(ops->tree->t, psi, m, pts, u, psi_at, (cudaStream_t)stream);
    });
}

int dafmm_nbody_direct(const dafmm_tree* tree, const double* v, double* out, void* stream)
{
    return guarded([&] {
        if (!tree || !v || !out) fail(DAFMM_EBADARG, "NULL argument");
        if (v == out) fail(DAFMM_EBADARG, "v and out must not overlap");
        require_device();
        nbody_direct(tree->t, v, out, (cudaStream_t)stream);
    });
}

int tree_info(const dafmm_tree* tree, dafmm_tree_info* info)
{
    return guarded([&] {
        if (!tree || !info) fail(DAFMM_EBADARG, "NULL argument");
        const Tree& t = tree->t;
        std::memset(info, 0, sizeof(*info));
        info->N = t.N;
        info->n_side = t.n_side;
        info->levels = t.L + 1;
        info->top = t.top;
        for (int nu = 0; nu <= t.L && nu < 32; nu++) {
            info->hf[nu] = t.lv[nu].hf;
            info->cones[nu] = t.lv[nu].nc;
            info->il_pairs[nu] = t.lv[nu].il_idx.size();
        }
    });
}

int tree_check(const dafmm_tree* tree, long* bad)
{
    return guarded([&] {
        if (!tree || !bad) fail(DAFMM_EBADARG, "NULL argument");
        *bad = check_tree(tree->t);
    });
}

int tree_destroy(dafmm_tree* tree)
{
    delete tree;
    return DAFMM_OK;
}

int build_nca_operators(dafmm_tree* tree, const double* q_dev, void* stream, dafmm_ops** out)
{
    dafmm_ops* ops = nullptr;
    int st = guarded([&] {
        if (!tree || !q_dev || !out) fail(DAFMM_EBADARG, "NULL argument");
        *out = nullptr;
        require_device();
        const Tree& t = tree->t;
        ops = new dafmm_ops();
        ops->tree = tree;
        double t_tab = build_entry_table(t, ops->table, stream);
        OpsHost h;
        build_nca(t, ops->table, h);
        fill_stats(t, h, ops->stats);
        ops->stats.setup_seconds_table = t_tab;
        ops->stats.setup_seconds_nca = h.t_nca;
        upload_ops(t, h, ops->dev);
        ops->stats.launches_per_call = launches_per_call(t, ops->dev, DAFMM_MIXED);
        ops->stats.launches_per_call_fp64 = launches_per_call(t, ops->dev, DAFMM_FP64);
        ops->stats.cmacs_far_fused = ops->dev.fz.cmacs;
        ops->stats.cmacs_leaf_fused = ops->dev.fz.leaf_cmacs;
        double* q = nullptr;
        if (cudaMalloc(&q, sizeof(double) * t.N) != cudaSuccess) {
            cudaGetLastError();
            fail(DAFMM_ENOMEM, "device allocation for q failed");
        }
        ops->dev.q = q;
        cudaError_t e = cudaMemcpyAsync(q, q_dev, sizeof(double) * t.N, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) fail(DAFMM_ECUDA, std::string("copy of q: ") + cudaGetErrorString(e));
        *out = ops;
    });
    if (st != DAFMM_OK && ops) {
        free_ops(ops->dev);
        delete ops;
    }
    return st;
}

int dafmm_matvec(const dafmm_ops* ops, int nrhs, const double* v, double* out, int precision, void* stream)
{
    return guarded([&] {
        if (!ops || !v || !out) fail(DAFMM_EBADARG, "NULL argument");
        if (nrhs < 1) fail(DAFMM_EBADARG, "nrhs must be >= 1");
        if (precision != DAFMM_FP64 && precision != DAFMM_MIXED) fail(DAFMM_EBADARG, "unknown precision");
        if (v == out) fail(DAFMM_EBADARG, "v and out must not overlap");
        apply_matvec(ops->tree->t, const_cast<dafmm_ops*>(ops)->dev, nrhs, v, out, precision, (cudaStream_t)stream);
    });
}

int dafmm_potential(const dafmm_ops* ops, int nrhs, const double* v, double* out, int precision, void* stream)
{
    return guarded([&] {
        if (!ops || !v || !out) fail(DAFMM_EBADARG, "NULL argument");
        if (nrhs < 1) fail(DAFMM_EBADARG, "nrhs must be >= 1");
        if (precision != DAFMM_FP64 && precision != DAFMM_MIXED) fail(DAFMM_EBADARG, "unknown precision");
        if (v == out) fail(DAFMM_EBADARG, "v and out must not overlap");
        apply_potential(ops->tree->t, const_cast<dafmm_ops*>(ops)->dev, nrhs, v, out, precision, (cudaStream_t)stream);
    });
}

int dafmm_matvec_noalloc(const dafmm_ops* ops, const double* v, double* out, int precision, void* stream)
{
    return guarded([&] {
        if (!ops || !v || !out) fail(DAFMM_EBADARG, "NULL argument");
        if (precision != DAFMM_FP64 && precision != DAFMM_MIXED) fail(DAFMM_EBADARG, "unknown precision");
        if (v == out) fail(DAFMM_EBADARG, "v and out must not overlap");
        apply_matvec_noalloc(ops->tree->t, ops->dev, v, out, precision, (cudaStream_t)stream);
    });
}

namespace {
void cuda_check(cudaError_t e, const char* what)
{
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(DAFMM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

void check_gmres(const dafmm_ops* ops, const double* f, const double* x, const gmres_opts* opts, const gmres_stats* st)
{
    if (!ops || !f || !x || !opts || !st) fail(DAFMM_EBADARG, "NULL argument");
    if (opts->restart < 1 || opts->restart > 128) fail(DAFMM_EBADARG, "restart must lie in 1..128");
    if (opts->max_iters < 0) fail(DAFMM_EBADARG, "max_iters must be >= 0");
    if (!(opts->tol > 0)) fail(DAFMM_EBADARG, "tol must be positive");
    if (opts->precision != DAFMM_FP64 && opts->precision != DAFMM_MIXED) fail(DAFMM_EBADARG, "unknown precision");
    if (opts->precision == DAFMM_MIXED && !(opts->inner_tol > 0 && opts->inner_tol < 1))
        fail(DAFMM_EBADARG, "inner_tol must lie in (0, 1) in mixed precision");
    for (int v : opts->reserved)
        if (v) fail(DAFMM_EBADARG, "reserved options must be zero");
    if (opts->side != DAFMM_PREC_RIGHT && opts->side != DAFMM_PREC_LEFT) fail(DAFMM_EBADARG, "side must be DAFMM_PREC_RIGHT or DAFMM_PREC_LEFT");
    if (f == x) fail(DAFMM_EBADARG, "f and x must not overlap");
}

// z = M^-1 v + alpha s N(q, v / s) (M^-1 = identity when M is NULL)
struct LearnedPrec {
    const dafmm_hodlr* M;
    dafmm_unet* net;
    const Tree* t;
    const OpsDev* d;
    double alpha;
    int applies;
};

void learned_prec(const void* P, const double* v, double* z, int precision, cudaStream_t s)
{
    auto* lp = (LearnedPrec*)P;
    if (lp->M)
        hodlr_prec(lp->M, v, z, precision, s);
    else
        cuda_check(cudaMemcpyAsync(z, v, sizeof(double2) * lp->t->N, cudaMemcpyDeviceToDevice, s), "cudaMemcpyAsync");
    unet_apply_nodes(lp->net, *lp->t, *lp->d, v, z, 1.0, lp->alpha, s);
    lp->applies++;
}
}  // namespace

int gmres_solve(dafmm_ops* ops, const dafmm_hodlr* M, int nrhs, const double* f, double* x, const gmres_opts* opts, gmres_stats* st,
                void* stream)
{
    int code = DAFMM_OK;
    int r = guarded([&] {
        check_gmres(ops, f, x, opts, st);
        if (nrhs < 1 || nrhs > 64) fail(DAFMM_EBADARG, "gmres_solve takes 1 to 64 right-hand sides");
        if (M && hodlr_tree(M) != ops->tree) fail(DAFMM_EBADARG, "the preconditioner was built on another tree");
        if (nrhs == 1)
            code = gmres_run(ops->tree->t, ops->dev, M, M ? hodlr_prec : nullptr, f, x, *opts, *st, (cudaStream_t)stream);
        else
            code = gmres_run_many(ops->tree->t, ops->dev, M, M ? hodlr_prec_many : nullptr, nrhs, f, x, *opts, st, (cudaStream_t)stream);
        if (M && hodlr_check(M, (cudaStream_t)stream) == DAFMM_ETIMEOUT)
            fail(DAFMM_ETIMEOUT, "a wait of the HODLR application gave up; the solution is undefined");
        if (code == DAFMM_ENOTCONV) {
            double worst = 0;
            for (int c = 0; c < nrhs; c++) worst = std::max(worst, st[c].rel_residual);
            fail(DAFMM_ENOTCONV, "GMRES reached max_iters at relative residual " + std::to_string(worst));
        }
    });
    return r;
}

int hodlr_factor(const dafmm_ops* ops, int rank, double tol, int leaf_size, dafmm_hodlr** out)
{
    return guarded([&] {
        if (!ops || !out) fail(DAFMM_EBADARG, "NULL argument");
        *out = nullptr;
        require_device();
        *out = hodlr_build(ops, rank, tol, leaf_size);
    });
}

int hodlr_solve(const dafmm_hodlr* M, int nrhs, const double* b, double* x, int precision, void* stream)
{
    return guarded([&] {
        if (!M || !b || !x) fail(DAFMM_EBADARG, "NULL argument");
        if (nrhs < 1 || nrhs > 64) fail(DAFMM_EBADARG, "hodlr_solve takes 1 to 64 right-hand sides");
        if (precision != DAFMM_FP64 && precision != DAFMM_MIXED) fail(DAFMM_EBADARG, "unknown precision");
        if (nrhs == 1)
            hodlr_apply(M, b, x, precision, (cudaStream_t)stream);
        else
            hodlr_apply_many(M, nrhs, b, x, precision, (cudaStream_t)stream);
    });
}

int hodlr_sync(const dafmm_hodlr* M, void* stream)
{
    return guarded([&] {
        if (!M) fail(DAFMM_EBADARG, "NULL argument");
        if (hodlr_check(M, (cudaStream_t)stream) == DAFMM_ETIMEOUT)
            fail(DAFMM_ETIMEOUT, "a grid barrier of the HODLR application gave up");
    });
}

int hodlr_set_ctas(dafmm_hodlr* M, int ctas)
{
    return guarded([&] {
        if (!M) fail(DAFMM_EBADARG, "NULL argument");
        hodlr_set_width(M, ctas);
    });
}

int hodlr_debug_stall(const dafmm_hodlr* M)
{
    return guarded([&] {
        if (!M) fail(DAFMM_EBADARG, "NULL argument");
        hodlr_set_stall(M, 1);
    });
}

int hodlr_export(const dafmm_hodlr* M, double* dense)
{
    return guarded([&] {
        if (!M || !dense) fail(DAFMM_EBADARG, "NULL argument");
        hodlr_dense(M, (cd*)dense);
    });
}

int hodlr_info(const dafmm_hodlr* M, long* N, int* levels, int* leaf_size, int* rank_max, double* seconds)
{
    return guarded([&] {
        if (!M || !N || !levels || !leaf_size || !rank_max || !seconds) fail(DAFMM_EBADARG, "NULL argument");
        hodlr_shape(M, N, levels, leaf_size, rank_max, seconds);
    });
}

int hodlr_destroy(dafmm_hodlr* M)
{
    hodlr_free(M);
    return DAFMM_OK;
}

int dafmm_sync(dafmm_ops* ops, void* stream)
{
    int st = DAFMM_OK;
    int r = guarded([&] {
        if (!ops) fail(DAFMM_EBADARG, "NULL argument");
        st = sync_and_check(ops->dev, (cudaStream_t)stream);
        if (st == DAFMM_ETIMEOUT) fail(DAFMM_ETIMEOUT, "a device-side wait gave up (a bulk copy or a tree pass did not arrive in time)");
    });
    return r;
}

int dafmm_set_batched_kernel(dafmm_ops* ops, int mode)
{
    return guarded([&] {
        if (!ops) fail(DAFMM_EBADARG, "NULL argument");
        set_batched_kernel(ops->dev, mode);
    });
}

int dafmm_set_batched_grid(dafmm_ops* ops, int ctas_per_sm)
{
    return guarded([&] {
        if (!ops) fail(DAFMM_EBADARG, "NULL argument");
        set_batched_grid(ops->dev, ctas_per_sm);
    });
}

int dafmm_tune_batched(dafmm_ops* ops, int nrhs, int precision, dafmm_tuning* out)
{
    return guarded([&] {
        if (!ops || !out) fail(DAFMM_EBADARG, "NULL argument");
        if (nrhs < 2 || nrhs > 64) fail(DAFMM_EBADARG, "nrhs must lie in 2..64");
        if (precision != DAFMM_FP64 && precision != DAFMM_MIXED) fail(DAFMM_EBADARG, "unknown precision");
        require_device();
        std::memset(out, 0, sizeof(*out));
        tune_batched(ops, nrhs, precision, *out);
    });
}

int dafmm_batch_create(int n, dafmm_ops* const* ops, dafmm_batch** out)
{
    return guarded([&] {
        if (!ops || !out || n < 1) fail(DAFMM_EBADARG, "NULL argument or no problems");
        *out = nullptr;
        for (int i = 0; i < n; i++)
            if (!ops[i]) fail(DAFMM_EBADARG, "NULL operator in the batch");
        require_device();
        *out = batch_new(n, ops);
    });
}

int dafmm_batch_matvec(dafmm_batch* b, int nrhs, const double* const* v, double* const* out, int precision, void* stream)
{
    return guarded([&] {
        if (!b || !v || !out) fail(DAFMM_EBADARG, "NULL argument");
        if (nrhs < 1 || nrhs > 64) fail(DAFMM_EBADARG, "nrhs must lie in 1..64");
        if (precision != DAFMM_FP64 && precision != DAFMM_MIXED) fail(DAFMM_EBADARG, "unknown precision");
        const size_t n = batch_size(b);
        for (size_t i = 0; i < n; i++)
            if (!v[i] || !out[i] || v[i] == out[i]) fail(DAFMM_EBADARG, "NULL or aliased vector in the batch");
        batch_matvec(b, nrhs, v, out, precision, (cudaStream_t)stream);
    });
}

int dafmm_batch_destroy(dafmm_batch* b)
{
    batch_free(b);
    return DAFMM_OK;
}

int dafmm_set_contrast(dafmm_ops* ops, const double* q_dev, void* stream)
{
    return guarded([&] {
        if (!ops || !q_dev) fail(DAFMM_EBADARG, "NULL argument");
        cuda_check(cudaMemcpyAsync(ops->dev.q, q_dev, sizeof(double) * ops->tree->t.N, cudaMemcpyDeviceToDevice, (cudaStream_t)stream),
                   "copy of q");
    });
}

int dafmm_debug_stall(dafmm_ops* ops, int pass)
{
    return guarded([&] {
        if (!ops) fail(DAFMM_EBADARG, "NULL argument");
        if (pass < -1 || pass >= (int)ops->dev.fz.g.passes.size()) fail(DAFMM_EBADARG, "pass out of range");
        ops->dev.stall_pass = pass;
    });
}

int dafmm_debug_leaf_staging(dafmm_ops* ops, int enable)
{
    return guarded([&] {
        if (!ops) fail(DAFMM_EBADARG, "NULL argument");
        if (enable != 0 && enable != 1) fail(DAFMM_EBADARG, "enable must be 0 or 1");
        set_leaf_staging(ops->dev, enable == 1);
    });
}

int dafmm_stats(const dafmm_ops* ops, dafmm_stats_t* stats)
{
    return guarded([&] {
        if (!ops || !stats) fail(DAFMM_EBADARG, "NULL argument");
        *stats = ops->stats;
    });
}

int dafmm_entries(const dafmm_ops* ops, long nr, const long* rows, long nc, const long* cols, double* out)
{
    return guarded([&] {
        if (!ops || (nr && !rows) || (nc && !cols) || (nr && nc && !out)) fail(DAFMM_EBADARG, "NULL argument");
        const long N = ops->tree->t.N;
        for (long a = 0; a < nr; a++)
            if (rows[a] < 0 || rows[a] >= N) fail(DAFMM_EBADARG, "row index out of range");
        for (long b = 0; b < nc; b++)
            if (cols[b] < 0 || cols[b] >= N) fail(DAFMM_EBADARG, "column index out of range");
        for (long a = 0; a < nr; a++)
            for (long b = 0; b < nc; b++) {
                cd v = ops->table(rows[a], cols[b]);
                out[2 * (a * nc + b)] = v.real();
                out[2 * (a * nc + b) + 1] = v.imag();
            }
    });
}

int dafmm_profile(dafmm_ops* ops, int enable)
{
    return guarded([&] {
        if (!ops) fail(DAFMM_EBADARG, "NULL argument");
        profile_enable(ops->dev, enable != 0);
    });
}

int dafmm_profile_read(dafmm_ops* ops, dafmm_profile_t* out)
{
    return guarded([&] {
        if (!ops || !out) fail(DAFMM_EBADARG, "NULL argument");
        profile_read(ops->dev, *out);
    });
}

int ops_destroy(dafmm_ops* ops)
{
    if (!ops) return DAFMM_OK;
    free_ops(ops->dev);
    delete ops;
    return DAFMM_OK;
}

int unet_create(const unet_params* p, dafmm_unet** out)
{
    return guarded([&] {
        if (!p || !out) fail(DAFMM_EBADARG, "NULL argument");
        *out = nullptr;
        for (int v : p->reserved)
            if (v) fail(DAFMM_EBADARG, "reserved parameters must be zero");
        require_device();
        *out = unet_new(*p);
    });
}

int unet_destroy(dafmm_unet* net)
{
    return guarded([&] { unet_delete(net); });
}

int unet_num_params(const dafmm_unet* net, long* n)
{
    return guarded([&] {
        if (!net || !n) fail(DAFMM_EBADARG, "NULL argument");
        *n = unet_size(net);
    });
}

int unet_get_params(const dafmm_unet* net, float* host)
{
    return guarded([&] {
        if (!net || !host) fail(DAFMM_EBADARG, "NULL argument");
        unet_get(net, host);
    });
}

int unet_set_params(dafmm_unet* net, const float* host)
{
    return guarded([&] {
        if (!net || !host) fail(DAFMM_EBADARG, "NULL argument");
        unet_set(net, host);
    });
}

int unet_forward(dafmm_unet* net, int batch, int height, int width, const float* in, float* out, void* stream)
{
    return guarded([&] {
        if (!net || !in || !out) fail(DAFMM_EBADARG, "NULL argument");
        unet_fwd(net, batch, height, width, in, out, (cudaStream_t)stream);
    });
}

int unet_backward(dafmm_unet* net, int batch, int height, int width, const float* in, const float* target, float* out, double* loss,
                  void* stream)
{
    return guarded([&] {
        if (!net || !in || !target || !out || !loss) fail(DAFMM_EBADARG, "NULL argument");
        *loss = unet_bwd(net, batch, height, width, in, target, out, (cudaStream_t)stream);
    });
}

int unet_get_grads(const dafmm_unet* net, float* host)
{
    return guarded([&] {
        if (!net || !host) fail(DAFMM_EBADARG, "NULL argument");
        unet_get_grad(net, host);
    });
}

int unet_adam(dafmm_unet* net, float lr, float beta1, float beta2, float eps, void* stream)
{
    return guarded([&] {
        if (!net) fail(DAFMM_EBADARG, "NULL argument");
        unet_adam_step(net, lr, beta1, beta2, eps, (cudaStream_t)stream);
    });
}

int unet_guess(dafmm_unet* net, const dafmm_ops* ops, const double* f, double* x, void* stream)
{
    return guarded([&] {
        if (!net || !ops || !f || !x) fail(DAFMM_EBADARG, "NULL argument");
        if (f == x) fail(DAFMM_EBADARG, "f and x must not overlap");
        unet_apply_nodes(net, ops->tree->t, ops->dev, f, x, 0.0, 1.0, (cudaStream_t)stream);
    });
}

int gmres_solve_learned(dafmm_ops* ops, const dafmm_hodlr* M, dafmm_unet* net, int flags, double alpha, const double* f, double* x,
                        const gmres_opts* opts, gmres_stats* st, learned_stats* ls, void* stream)
{
    int code = DAFMM_OK;
    double* tmp = nullptr;
    int r = guarded([&] {
        check_gmres(ops, f, x, opts, st);
        if (!net || !ls) fail(DAFMM_EBADARG, "NULL argument");
        if (flags & ~3) fail(DAFMM_EBADARG, "unknown flags");
        if ((flags & 2) && opts->side == DAFMM_PREC_LEFT)
            fail(DAFMM_EBADARG, "the coarse correction is a right preconditioner (side must be DAFMM_PREC_RIGHT)");
        if (M && hodlr_tree(M) != ops->tree) fail(DAFMM_EBADARG, "the preconditioner was built on another tree");
        const Tree& t = ops->tree->t;
        cudaStream_t s = (cudaStream_t)stream;
        ls->guess_used = 0;
        ls->guess_residual = -1;
        ls->corrections = 0;
        if (flags & 1) {
            // the network's guess, kept only if it beats x0 = 0
            if (cudaMalloc(&tmp, sizeof(double2) * 2 * t.N) != cudaSuccess) {
                cudaGetLastError();
                fail(DAFMM_ENOMEM, "device allocation for the guess failed");
            }
            unet_apply_nodes(net, t, ops->dev, f, tmp, 0.0, 1.0, s);
            ls->guess_residual = relative_residual(t, ops->dev, f, tmp, tmp + 2 * t.N, unet_scalars(net), s);
            if (ls->guess_residual < 1.0) {
                cuda_check(cudaMemcpyAsync(x, tmp, sizeof(double2) * t.N, cudaMemcpyDeviceToDevice, s), "cudaMemcpyAsync");
                ls->guess_used = 1;
            }
        }
        if (flags & 2) {
            LearnedPrec lp{M, net, &t, &ops->dev, alpha, 0};
            code = gmres_run(t, ops->dev, &lp, learned_prec, f, x, *opts, *st, s);
            ls->corrections = lp.applies;
        } else {
            code = gmres_run(t, ops->dev, M, M ? hodlr_prec : nullptr, f, x, *opts, *st, s);
        }
        if (M && hodlr_check(M, s) == DAFMM_ETIMEOUT)
            fail(DAFMM_ETIMEOUT, "a wait of the HODLR application gave up; the solution is undefined");
        if (code == DAFMM_ENOTCONV)
            fail(DAFMM_ENOTCONV, "GMRES reached max_iters at relative residual " + std::to_string(st->rel_residual));
    });
    cudaFree(tmp);
    return r;
}

}  // extern "C"
