// Partially pivoted adaptive cross approximation (Section 4.2.2 for the NCA
// pivots; also used for the HODLR off-diagonal blocks).
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace dafmm {

struct AcaPivots {
    std::vector<int> r, c;  // positions in the row and column lists
};

// ACA on the implicit matrix E(R[a], C[b]).  Stops when |u_k| |v_k| <=
// eps |S_k|_F with the Frobenius norm of the approximant updated recursively
// (Rjasanow); the pivot of that last update is not kept (the approximant
// before it already meets the tolerance, and a rounding-level pivot would make
// a skeleton's pivot block singular).  eps = 0 runs to maxr pivots (or until
// the residual vanishes).  Starts at the first row; the next row is the unused
// row of largest |u_k|, the pivot column the unused column of largest
// residual; ties go to the lowest index; a row whose residual vanishes is
// skipped for the next unused row.  If U and V are given they receive the
// kept factors: E ~= sum_k U[k] V[k]^T (U[k] over R, V[k] over C).
template <class Entry>
void aca_run(Entry E, const std::vector<long>& R, const std::vector<long>& C, double eps, int maxr, AcaPivots& out,
             std::vector<std::vector<cd>>* Uo, std::vector<std::vector<cd>>* Vo)
{
    const int m = (int)R.size(), n = (int)C.size();
    out.r.clear();
    out.c.clear();
    if (m == 0 || n == 0) return;
    int kmax = std::min(m, n);
    if (maxr > 0) kmax = std::min(kmax, maxr);
    std::vector<std::vector<cd>> U, V;
    std::vector<char> rused(m, 0), cused(n, 0);
    std::vector<cd> row(n), u(m);
    double s2 = 0.0, scale = 0.0;
    int i = 0;
    while ((int)out.r.size() < kmax) {
        for (int j = 0; j < n; j++) {
            cd a = E(R[i], C[j]);
            scale = std::max(scale, std::abs(a));
            for (size_t q = 0; q < U.size(); q++) a -= U[q][i] * V[q][j];
            row[j] = a;
        }
        rused[i] = 1;
        int jb = -1;
        double best = 0.0;
        for (int j = 0; j < n; j++)
            if (!cused[j] && std::abs(row[j]) > best) {
                best = std::abs(row[j]);
                jb = j;
            }
        if (jb < 0 || best <= 1e-15 * scale) {
            int nx = -1;
            for (int a = 0; a < m; a++)
                if (!rused[a]) {
                    nx = a;
                    break;
                }
            if (nx < 0) break;
            i = nx;
            continue;
        }
        const cd delta = row[jb];
        std::vector<cd> v(n);
        for (int j = 0; j < n; j++) v[j] = row[j] / delta;
        for (int a = 0; a < m; a++) {
            cd e = E(R[a], C[jb]);
            for (size_t q = 0; q < U.size(); q++) e -= U[q][a] * V[q][jb];
            u[a] = e;
        }
        cused[jb] = 1;
        out.r.push_back(i);
        out.c.push_back(jb);
        double nu2 = 0, nv2 = 0;
        for (int a = 0; a < m; a++) nu2 += std::norm(u[a]);
        for (int j = 0; j < n; j++) nv2 += std::norm(v[j]);
        for (size_t q = 0; q < U.size(); q++) {
            cd uu = 0, vv = 0;
            for (int a = 0; a < m; a++) uu += std::conj(U[q][a]) * u[a];
            for (int j = 0; j < n; j++) vv += std::conj(V[q][j]) * v[j];
            s2 += 2.0 * std::real(uu * vv);
        }
        s2 += nu2 * nv2;
        U.push_back(u);
        V.push_back(v);
        if (eps > 0 && std::sqrt(nu2 * nv2) <= eps * std::sqrt(std::max(s2, 0.0))) {
            out.r.pop_back();
            out.c.pop_back();
            U.pop_back();
            V.pop_back();
            break;
        }
        int nx = -1;
        double bu = -1.0;
        for (int a = 0; a < m; a++)
            if (!rused[a] && std::abs(u[a]) > bu) {
                bu = std::abs(u[a]);
                nx = a;
            }
        if (nx < 0) break;
        i = nx;
    }
    if (Uo) *Uo = std::move(U);
    if (Vo) *Vo = std::move(V);
}

}  // namespace dafmm
