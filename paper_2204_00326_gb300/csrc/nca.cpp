// Nested Cross Approximation setup (Section 4): nested pivots by partially
// pivoted ACA, the P2M/M2M and L2L/L2P operators of the four cases of
// Section 4.2.1, and the M2L blocks of Section 5 step 4.  Host code, OpenMP
// over the slots of one level; levels are processed from the leaves up.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "aca.h"
#include "internal.h"

namespace dafmm {
namespace {

AcaPivots aca(const EntryTable& K, const std::vector<long>& R, const std::vector<long>& C, double eps, int maxr)
{
    AcaPivots out;
    aca_run([&](long i, long j) { return K(i, j); }, R, C, eps, maxr, out, nullptr, nullptr);
    return out;
}

// LU with partial pivoting of an r x r complex matrix (row-major) and solves.
struct LU {
    int n = 0;
    std::vector<cd> a;
    std::vector<int> piv;
    bool factor(std::vector<cd> m, int nn)
    {
        n = nn;
        a = std::move(m);
        piv.resize(n);
        for (int c = 0; c < n; c++) {
            int p = c;
            double b = std::abs(a[c * n + c]);
            for (int r = c + 1; r < n; r++)
                if (std::abs(a[r * n + c]) > b) { b = std::abs(a[r * n + c]); p = r; }
            piv[c] = p;
            if (b == 0.0) return false;
            if (p != c)
                for (int k = 0; k < n; k++) std::swap(a[c * n + k], a[p * n + k]);
            cd inv = 1.0 / a[c * n + c];
            for (int r = c + 1; r < n; r++) {
                cd f = a[r * n + c] * inv;
                a[r * n + c] = f;
                if (f == cd(0)) continue;
                for (int k = c + 1; k < n; k++) a[r * n + k] -= f * a[c * n + k];
            }
        }
        return true;
    }
    // solve A x = b in place (b has n entries, stride 1)
    void solve(cd* b) const
    {
        // the multipliers moved with their rows, so apply every swap first
        for (int c = 0; c < n; c++)
            if (piv[c] != c) std::swap(b[c], b[piv[c]]);
        for (int c = 0; c < n; c++)
            for (int r = c + 1; r < n; r++) b[r] -= a[r * n + c] * b[c];
        for (int c = n - 1; c >= 0; c--) {
            cd s = b[c];
            for (int k = c + 1; k < n; k++) s -= a[c * n + k] * b[k];
            b[c] = s / a[c * n + c];
        }
    }
};

int pad_rank(int r)
{
    if (r <= 0) return 8;
    if (r <= 8) return 8;
    if (r <= 16) return 16;
    if (r <= 32) return 32;
    return (r + 15) / 16 * 16;
}

// Per-slot pivots and transfer blocks of one level.
struct SlotNCA {
    std::vector<long> t_in;   // t^{S,i}: incoming row (self) pivots, global point indices
    std::vector<long> s_out;  // s^{S,o}: outgoing column (self) pivots
    std::vector<cd> X;        // |t~in| x ri, row-major: incoming transfer (C blocks / U)
    std::vector<cd> Y;        // ro x |s~out|, row-major: outgoing transfer (T blocks / V*)
    std::vector<int> in_off, out_off;  // offsets of each child's block in t~in / s~out
    bool pass = false;
};

}  // namespace

void build_nca(const Tree& t, const EntryTable& K, OpsHost& ops)
{
    auto t0 = std::chrono::steady_clock::now();
    const int L = t.L;
    ops.lv.assign(L + 1, LevelOpsHost());

    // near-field blocks: source leaf at offset (sx, sy) from the target leaf,
    // block[(sy+1)*3 + (sx+1)][i'][j'] = K(target i', source j')
    ops.near.assign(9 * 256, cd(0));
    {
        const int nb = t.nb;
        for (int sy = -1; sy <= 1; sy++)
            for (int sx = -1; sx <= 1; sx++) {
                if (nb == 1 && (sx || sy)) continue;
                int dx = -sx + nb - 1, dy = -sy + nb - 1;
                if (dx < 0 || dy < 0 || dx > 2 * nb - 2 || dy > 2 * nb - 2) continue;
                const cd* src = &K.tab[((long)dy * (2 * nb - 1) + dx) * 256];
                std::copy(src, src + 256, &ops.near[((sy + 1) * 3 + (sx + 1)) * 256]);
            }
    }
    if (t.top > L) {
        ops.t_nca = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        return;
    }

    const double eps = t.prm.eps_nca;
    const int maxr = t.prm.max_rank;
    std::vector<std::vector<SlotNCA>> nca(L + 1);
    std::vector<int> ch;

    for (int nu = L; nu >= t.top; nu--) {
        const Level& l = t.lv[nu];
        auto& S = nca[nu];
        S.assign(l.nslot(), SlotNCA());
        const bool leaf = (nu == L);
        std::vector<int> err(l.nslot(), 0);
#pragma omp parallel for schedule(dynamic, 4)
        for (int s = 0; s < l.nslot(); s++) {
            if (!l.active[s]) continue;
            SlotNCA& me = S[s];
            std::vector<int> kids;
            std::vector<long> tin, sout;  // self candidates
            if (leaf) {
                for (int k = 0; k < 16; k++) {
                    tin.push_back((long)s * 16 + k);
                    sout.push_back((long)s * 16 + k);
                }
                me.in_off = {0, 16};
                me.out_off = {0, 16};
            } else {
                child_slots(t, nu, s, kids);
                me.in_off.push_back(0);
                me.out_off.push_back(0);
                for (int c : kids) {
                    const SlotNCA& cs = nca[nu + 1][c];
                    tin.insert(tin.end(), cs.t_in.begin(), cs.t_in.end());
                    sout.insert(sout.end(), cs.s_out.begin(), cs.s_out.end());
                    me.in_off.push_back((int)tin.size());
                    me.out_off.push_back((int)sout.size());
                }
            }
            // far candidates from the interaction list (Section 4.2.2, step 1)
            std::vector<long> sfar, tfar;
            std::vector<int> kk;
            for (int e = l.il_ptr[s]; e < l.il_ptr[s + 1]; e++) {
                int a = l.il_idx[e];
                if (leaf) {
                    for (int k = 0; k < 16; k++) {
                        sfar.push_back((long)a * 16 + k);
                        tfar.push_back((long)a * 16 + k);
                    }
                } else {
                    child_slots(t, nu, a, kk);
                    for (int c : kk) {
                        const SlotNCA& cs = nca[nu + 1][c];
                        sfar.insert(sfar.end(), cs.s_out.begin(), cs.s_out.end());
                        tfar.insert(tfar.end(), cs.t_in.begin(), cs.t_in.end());
                    }
                }
            }
            if (sfar.empty()) {
                // no list of its own but needed by an active parent: keep every
                // candidate (identity transfers)
                me.pass = true;
                me.t_in = tin;
                me.s_out = sout;
                int m = (int)tin.size(), n = (int)sout.size();
                me.X.assign((size_t)m * m, cd(0));
                for (int a = 0; a < m; a++) me.X[(size_t)a * m + a] = 1.0;
                me.Y.assign((size_t)n * n, cd(0));
                for (int a = 0; a < n; a++) me.Y[(size_t)a * n + a] = 1.0;
                continue;
            }
            // incoming: ACA on K(t~in, s~in) -> t^{S,i}, s^{S,i};
            // X = K(t~in, s^{S,i}) K(t^{S,i}, s^{S,i})^{-1}
            {
                AcaPivots pv = aca(K, tin, sfar, eps, maxr);
                const int r = (int)pv.r.size(), m = (int)tin.size();
                std::vector<cd> PT((size_t)r * r);  // P^T
                for (int a = 0; a < r; a++)
                    for (int b = 0; b < r; b++) PT[(size_t)b * r + a] = K(tin[pv.r[a]], sfar[pv.c[b]]);
                LU lu;
                if (!lu.factor(PT, r)) { err[s] = 1; continue; }
                me.X.assign((size_t)m * r, cd(0));
                std::vector<cd> rhs(r);
                for (int a = 0; a < m; a++) {
                    for (int b = 0; b < r; b++) rhs[b] = K(tin[a], sfar[pv.c[b]]);
                    lu.solve(rhs.data());  // P^T x = row^T  <=>  x^T = row P^{-1}
                    for (int b = 0; b < r; b++) me.X[(size_t)a * r + b] = rhs[b];
                }
                for (int a = 0; a < r; a++) me.t_in.push_back(tin[pv.r[a]]);
            }
            // outgoing: ACA on K(t~out, s~out) -> t^{S,o}, s^{S,o};
            // Y = K(t^{S,o}, s^{S,o})^{-1} K(t^{S,o}, s~out)
            {
                AcaPivots pv = aca(K, tfar, sout, eps, maxr);
                const int r = (int)pv.r.size(), n = (int)sout.size();
                std::vector<cd> P((size_t)r * r);
                for (int a = 0; a < r; a++)
                    for (int b = 0; b < r; b++) P[(size_t)a * r + b] = K(tfar[pv.r[a]], sout[pv.c[b]]);
                LU lu;
                if (!lu.factor(P, r)) { err[s] = 1; continue; }
                me.Y.assign((size_t)r * n, cd(0));
                std::vector<cd> col(r);
                for (int j = 0; j < n; j++) {
                    for (int a = 0; a < r; a++) col[a] = K(tfar[pv.r[a]], sout[j]);
                    lu.solve(col.data());
                    for (int a = 0; a < r; a++) me.Y[(size_t)a * n + j] = col[a];
                }
                for (int b = 0; b < r; b++) me.s_out.push_back(sout[pv.c[b]]);
            }
        }
        for (int s = 0; s < l.nslot(); s++)
            if (err[s]) fail(DAFMM_EBREAKDOWN, "singular NCA pivot block at level " + std::to_string(nu));

        LevelOpsHost& lo = ops.lv[nu];
        lo.ri.assign(l.nslot(), 0);
        lo.ro.assign(l.nslot(), 0);
        int rimax = 0, romax = 0;
        for (int s = 0; s < l.nslot(); s++) {
            lo.ri[s] = (int)S[s].t_in.size();
            lo.ro[s] = (int)S[s].s_out.size();
            rimax = std::max(rimax, lo.ri[s]);
            romax = std::max(romax, lo.ro[s]);
        }
        lo.Ri = pad_rank(rimax);
        lo.Ro = pad_rank(romax);
    }

    // ---- assemble block-sparse operators at the realised ranks ----
    for (int nu = t.top; nu <= L; nu++) {
        const Level& l = t.lv[nu];
        LevelOpsHost& lo = ops.lv[nu];
        const auto& S = nca[nu];
        const bool leaf = (nu == L);

        // M2L: rows slots of nu, entries the interaction list, blocks K(t^{S,i}, s^{S',o})
        {
            BsrHost& b = lo.m2l;
            b.nrows = l.nslot();
            b.Rout = lo.Ri;
            b.Rin = lo.Ro;
            b.rout = lo.ri;
            b.rowptr.assign(b.nrows + 1, 0);
            for (int s = 0; s < l.nslot(); s++) b.rowptr[s + 1] = b.rowptr[s] + (l.active[s] ? l.il_ptr[s + 1] - l.il_ptr[s] : 0);
            b.col.resize(b.rowptr.back());
            b.rin.resize(b.rowptr.back());
            for (int s = 0; s < l.nslot(); s++) {
                if (!l.active[s]) continue;
                for (int e = l.il_ptr[s]; e < l.il_ptr[s + 1]; e++) {
                    long k = b.rowptr[s] + (e - l.il_ptr[s]);
                    b.col[k] = l.il_idx[e];
                    b.rin[k] = lo.ro[l.il_idx[e]];
                }
            }
            b.layout();
#pragma omp parallel for schedule(dynamic, 8)
            for (int s = 0; s < l.nslot(); s++) {
                const auto& ti = S[s].t_in;
                const size_t ldr = b.ld[s];
                for (int k = b.rowptr[s]; k < b.rowptr[s + 1]; k++) {
                    cd* M = &b.mats[b.moff[k]];
                    const auto& so = S[b.col[k]].s_out;
                    for (size_t jj = 0; jj < so.size(); jj++)
                        for (size_t ii = 0; ii < ti.size(); ii++) M[jj * ldr + ii] = K(ti[ii], so[jj]);
                }
            }
        }
        // UP (P2M at the leaves, M2M above): rows slots of nu, blocks T (ro x ro_child) / V* (ro x 16)
        {
            BsrHost& b = lo.up;
            b.nrows = l.nslot();
            b.Rout = lo.Ro;
            b.Rin = leaf ? 16 : ops.lv[nu + 1].Ro;
            b.rout = lo.ro;
            b.rowptr.assign(b.nrows + 1, 0);
            std::vector<std::vector<int>> cols(b.nrows);
            for (int s = 0; s < l.nslot(); s++) {
                if (!l.active[s]) continue;
                if (leaf)
                    cols[s] = {s};
                else
                    child_slots(t, nu, s, cols[s]);
                b.rowptr[s + 1] = (int)cols[s].size();
            }
            for (int s = 0; s < b.nrows; s++) b.rowptr[s + 1] += b.rowptr[s];
            b.col.resize(b.rowptr.back());
            b.rin.resize(b.rowptr.back());
            for (int s = 0; s < l.nslot(); s++)
                for (size_t c = 0; c < cols[s].size(); c++) {
                    long e = b.rowptr[s] + (long)c;
                    b.col[e] = cols[s][c];
                    b.rin[e] = leaf ? 16 : ops.lv[nu + 1].ro[cols[s][c]];
                }
            b.layout();
            for (int s = 0; s < l.nslot(); s++) {
                if (!l.active[s]) continue;
                const SlotNCA& me = S[s];
                const int ro = (int)me.s_out.size();
                const int ncand = me.out_off.back();
                for (size_t c = 0; c < cols[s].size(); c++) {
                    long e = b.rowptr[s] + (long)c;
                    cd* M = &b.mats[b.moff[e]];
                    for (int j = me.out_off[c]; j < me.out_off[c + 1]; j++)
                        for (int a = 0; a < ro; a++) M[(size_t)(j - me.out_off[c]) * b.ld[s] + a] = me.Y[(size_t)a * ncand + j];
                }
            }
        }
        // DOWN (L2L to nu+1, or L2P at the leaves): rows slots of nu+1 / leaves
        {
            BsrHost& b = lo.down;
            if (leaf) {
                b.nrows = l.nslot();
                b.Rout = 16;
                b.Rin = lo.Ri;
                b.rout.assign(b.nrows, 16);
                b.rowptr.assign(b.nrows + 1, 0);
                for (int s = 0; s < l.nslot(); s++) b.rowptr[s + 1] = b.rowptr[s] + (l.active[s] ? 1 : 0);
                b.col.resize(b.rowptr.back());
                b.rin.resize(b.rowptr.back());
                for (int s = 0; s < l.nslot(); s++)
                    if (l.active[s]) {
                        b.col[b.rowptr[s]] = s;
                        b.rin[b.rowptr[s]] = lo.ri[s];
                    }
                b.layout();
                for (int s = 0; s < l.nslot(); s++) {
                    if (!l.active[s]) continue;
                    const SlotNCA& me = S[s];
                    const int ri = (int)me.t_in.size();
                    cd* M = &b.mats[b.moff[b.rowptr[s]]];
                    for (int jj = 0; jj < ri; jj++)
                        for (int a = 0; a < 16; a++) M[(size_t)jj * 16 + a] = me.X[(size_t)a * ri + jj];
                }
            } else {
                const Level& lc = t.lv[nu + 1];
                const LevelOpsHost& loc = ops.lv[nu + 1];
                b.nrows = lc.nslot();
                b.Rout = loc.Ri;
                b.Rin = lo.Ri;
                b.rout = loc.ri;
                std::vector<std::vector<std::pair<int, int>>> ent(b.nrows);  // (parent slot, child position)
                for (int s = 0; s < l.nslot(); s++) {
                    if (!l.active[s]) continue;
                    std::vector<int> kids;
                    child_slots(t, nu, s, kids);
                    for (size_t c = 0; c < kids.size(); c++) ent[kids[c]].push_back({s, (int)c});
                }
                b.rowptr.assign(b.nrows + 1, 0);
                for (int r = 0; r < b.nrows; r++) b.rowptr[r + 1] = b.rowptr[r] + (int)ent[r].size();
                b.col.resize(b.rowptr.back());
                b.rin.resize(b.rowptr.back());
                for (int r = 0; r < b.nrows; r++)
                    for (size_t k = 0; k < ent[r].size(); k++) {
                        b.col[b.rowptr[r] + k] = ent[r][k].first;
                        b.rin[b.rowptr[r] + k] = lo.ri[ent[r][k].first];
                    }
                b.layout();
#pragma omp parallel for schedule(dynamic, 16)
                for (int r = 0; r < b.nrows; r++) {
                    const int rc = b.ld[r];
                    for (size_t k = 0; k < ent[r].size(); k++) {
                        long e = b.rowptr[r] + (long)k;
                        int s = ent[r][k].first, c = ent[r][k].second;
                        const SlotNCA& me = S[s];
                        const int ri = (int)me.t_in.size();
                        cd* M = &b.mats[b.moff[e]];
                        for (int a = me.in_off[c]; a < me.in_off[c + 1]; a++)
                            for (int jj = 0; jj < ri; jj++) M[(size_t)jj * rc + (a - me.in_off[c])] = me.X[(size_t)a * ri + jj];
                    }
                }
            }
        }
    }
    ops.t_nca = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace dafmm
