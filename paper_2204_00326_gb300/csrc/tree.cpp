// Uniform quadtree, regimes, cones and interaction lists (Sections 3, 4.1, Table 1).
#include <algorithm>
#include <cmath>
#include <cstring>

#include <unordered_set>

#include "internal.h"

namespace dafmm {

long morton_encode(int x, int y)
{
    long m = 0;
    for (int k = 0; k < 31; k++) {
        m |= (long)((x >> k) & 1) << (2 * k);
        m |= (long)((y >> k) & 1) << (2 * k + 1);
    }
    return m;
}

void morton_decode(long m, int* x, int* y)
{
    int xx = 0, yy = 0;
    for (int k = 0; k < 31; k++) {
        xx |= (int)((m >> (2 * k)) & 1) << k;
        yy |= (int)((m >> (2 * k + 1)) & 1) << k;
    }
    *x = xx;
    *y = yy;
}

void cheb_nodes(int p, double* z)
{
    // z_k = -cos((2k+1) pi / (2p)): first-kind nodes, ascending
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < p; k++) z[k] = -std::cos((2 * k + 1) * pi / (2.0 * p));
}

namespace {

const long double kTwoPi = 6.283185307179586476925286766559L;

// Same-level neighbours (Table 1).  Low frequency: boxes that are not
// well separated, i.e. centres closer than 4w (Section 3.1): |d|_inf <= 1 in
// box units.  High frequency: boxes that violate the distance condition
// |x - y| >= kappa w^2 of the directional admissibility (Section 3.2).
bool is_neighbor(const Level& l, double kappa, long dx, long dy)
{
    if (!l.hf) return std::max(std::labs(dx), std::labs(dy)) <= 1;
    double d = 2.0 * l.w * std::sqrt((double)(dx * dx + dy * dy));
    return d < kappa * l.w * l.w * (1.0 - 1e-12);
}

// Cone containing direction (dx, dy) among nc cones [2 pi j/nc, 2 pi (j+1)/nc).
// A direction on a boundary belongs to the cone that starts there.
int cone_of(long dx, long dy, int nc)
{
    long double th = atan2l((long double)dy, (long double)dx);
    if (th < 0) th += kTwoPi;
    long double x = th * nc / kTwoPi;
    long double k = floorl(x + 0.5L);
    long c;
    if (fabsl(x - k) < 1e-9L)
        c = (long)k;
    else
        c = (long)floorl(x);
    return (int)(((c % nc) + nc) % nc);
}

// Neighbour radius (box units) worth scanning at level l.
long scan_radius(const Level& l, double kappa)
{
    if (!l.hf) return 1;
    double r = kappa * l.w / 2.0;
    return std::min<long>((long)std::ceil(r) + 1, l.nside);
}

}  // namespace

void child_slots(const Tree& t, int nu, int s, std::vector<int>& out)
{
    out.clear();
    const Level& P = t.lv[nu];
    const Level& C = t.lv[nu + 1];
    if (!P.hf) {
        for (int c = 0; c < 4; c++) out.push_back(4 * s + c);
        return;
    }
    int box = s / P.nc, cone = s % P.nc;
    if (!C.hf) {
        for (int c = 0; c < 4; c++) out.push_back(4 * box + c);
    } else {
        // the parent's cone is inside cone floor(cone/2) of every child (Section 3.2.1)
        for (int c = 0; c < 4; c++) out.push_back((4 * box + c) * C.nc + cone / 2);
    }
}

Tree* make_tree(const dafmm_params& prm, int n_side, double x0, double x1)
{
    if (prm.p != 4) fail(DAFMM_EBADARG, "only p = 4 nodes per leaf side is supported");
    if (!(prm.kappa > 0)) fail(DAFMM_EBADARG, "kappa must be positive");
    if (!(prm.eps_nca > 0 && prm.eps_nca < 1)) fail(DAFMM_EBADARG, "eps_nca must lie in (0, 1)");
    if (!(prm.T > 0)) fail(DAFMM_EBADARG, "T must be positive");
    if (prm.max_rank < 0) fail(DAFMM_EBADARG, "max_rank must be >= 0");
    if (prm.kernel != DAFMM_KERNEL_LS && prm.kernel != DAFMM_KERNEL_POINTS)
        fail(DAFMM_EBADARG, "kernel must be DAFMM_KERNEL_LS or DAFMM_KERNEL_POINTS");
    for (int r : prm.reserved)
        if (r) fail(DAFMM_EBADARG, "reserved parameters must be zero");
    if (!(x1 > x0)) fail(DAFMM_EBADARG, "x1 must exceed x0");
    if (n_side < prm.p || n_side % prm.p) fail(DAFMM_EBADARG, "n_side must be a positive multiple of p");
    int nb = n_side / prm.p;
    if (nb & (nb - 1)) fail(DAFMM_EBADARG, "n_side / p must be a power of two");
    if (nb > (1 << 14)) fail(DAFMM_EBADARG, "grid too large");

    Tree* t = new Tree();
    t->prm = prm;
    t->n_side = n_side;
    t->p = prm.p;
    t->nb = nb;
    int L = 0;
    while ((1 << L) < nb) L++;
    t->L = L;
    t->N = (long)n_side * n_side;
    t->x0 = x0;
    t->x1 = x1;
    t->beta = (x1 - x0) / (2.0 * nb);
    const double kappa = prm.kappa;

    t->lv.resize(L + 1);
    int finest_hf = -1;
    for (int nu = 0; nu <= L; nu++) {
        Level& l = t->lv[nu];
        l.nu = nu;
        l.nside = 1 << nu;
        l.nbox = l.nside * l.nside;
        l.w = (x1 - x0) / (double)(2 << nu);
        l.hf = (kappa * l.w) * (kappa * l.w) > prm.T;
        if (l.hf) finest_hf = nu;
    }
    if (t->lv[L].hf) {
        delete t;
        fail(DAFMM_EBADARG, "leaf boxes are in the high-frequency regime; refine the grid");
    }
    if (finest_hf >= 0) {
        // cone angle 2 pi / nc <= 1 / (kappa w) at the finest high-frequency
        // level, doubling the count per level up (Section 3.2, 3.2.1)
        double want = 2.0 * M_PI * kappa * t->lv[finest_hf].w;
        int nc = 1;
        while (nc < want) nc <<= 1;
        nc = std::max(nc, 4);
        for (int nu = finest_hf; nu >= 0; nu--) {
            long c = (long)nc << (finest_hf - nu);
            if (c > (1 << 20)) c = 1 << 20;
            t->lv[nu].nc = (int)c;
        }
    }

    for (int l = 0; l < nb * nb; l++) {
        int x, y;
        morton_decode(l, &x, &y);
        t->leaf_x.push_back(x);
        t->leaf_y.push_back(y);
    }

    // Interaction lists: children of the parent's neighbours that are not
    // neighbours (Table 1), split by cone at high-frequency levels.
    std::vector<std::vector<int>> il;
    t->top = L + 1;
    for (int nu = 1; nu <= L; nu++) {
        Level& l = t->lv[nu];
        const Level& par = t->lv[nu - 1];
        il.assign(l.nslot(), {});
        long prad = scan_radius(par, kappa);
        long pairs = 0;
        for (int b = 0; b < l.nbox; b++) {
            int bx, by;
            morton_decode(b, &bx, &by);
            int px = bx >> 1, py = by >> 1;
            for (long ddy = -prad; ddy <= prad; ddy++)
                for (long ddx = -prad; ddx <= prad; ddx++) {
                    long qx = px + ddx, qy = py + ddy;
                    if (qx < 0 || qy < 0 || qx >= par.nside || qy >= par.nside) continue;
                    if (!is_neighbor(par, kappa, ddx, ddy)) continue;
                    for (int c = 0; c < 4; c++) {
                        long ax = 2 * qx + (c & 1), ay = 2 * qy + (c >> 1);
                        long dx = ax - bx, dy = ay - by;
                        if (is_neighbor(l, kappa, dx, dy)) continue;
                        int a = (int)morton_encode((int)ax, (int)ay);
                        if (!l.hf) {
                            il[b].push_back(a);
                        } else {
                            int cl = cone_of(dx, dy, l.nc);
                            int cr = cone_of(-dx, -dy, l.nc);
                            il[(long)b * l.nc + cl].push_back(a * l.nc + cr);
                        }
                        pairs++;
                    }
                }
        }
        l.il_ptr.assign(l.nslot() + 1, 0);
        for (int s = 0; s < l.nslot(); s++) {
            std::sort(il[s].begin(), il[s].end());
            l.il_ptr[s + 1] = l.il_ptr[s] + (int)il[s].size();
        }
        l.il_idx.resize(l.il_ptr.back());
        for (int s = 0; s < l.nslot(); s++) std::copy(il[s].begin(), il[s].end(), l.il_idx.begin() + l.il_ptr[s]);
        if (pairs > 0 && t->top > L) t->top = nu;
    }
    t->lv[0].il_ptr.assign(t->lv[0].nslot() + 1, 0);

    // Active slots: own list non-empty, or a related slot one level up is active.
    for (int nu = 0; nu <= L; nu++) t->lv[nu].active.assign(t->lv[nu].nslot(), 0);
    std::vector<int> ch;
    for (int nu = t->top; nu <= L; nu++) {
        Level& l = t->lv[nu];
        for (int s = 0; s < l.nslot(); s++)
            if (l.il_ptr[s + 1] > l.il_ptr[s]) l.active[s] = 1;
        if (nu > t->top) {
            const Level& par = t->lv[nu - 1];
            for (int s = 0; s < par.nslot(); s++) {
                if (!par.active[s]) continue;
                child_slots(*t, nu - 1, s, ch);
                for (int c : ch) l.active[c] = 1;
            }
        }
    }
    return t;
}

long check_tree(const Tree& t)
{
    long bad = 0;
    const int L = t.L, nb = t.nb;
    // IL pairs per level as (target box, source box) with multiplicity
    std::vector<std::unordered_multiset<long>> pairs(L + 1);
    for (int nu = 1; nu <= L; nu++) {
        const Level& l = t.lv[nu];
        std::unordered_set<long> entries;
        for (int s = 0; s < l.nslot(); s++)
            for (int e = l.il_ptr[s]; e < l.il_ptr[s + 1]; e++) {
                int a = l.il_idx[e];
                pairs[nu].insert((long)(s / l.nc) * l.nbox + a / l.nc);
                entries.insert((long)s * l.nslot() + a);
            }
        if (l.hf)
            for (int s = 0; s < l.nslot(); s++)
                for (int e = l.il_ptr[s]; e < l.il_ptr[s + 1]; e++)
                    if (!entries.count((long)l.il_idx[e] * l.nslot() + s)) bad++;
    }
    for (int a = 0; a < nb * nb; a++)
        for (int b = 0; b < nb * nb; b++) {
            int cover = (std::max(std::abs(t.leaf_x[a] - t.leaf_x[b]), std::abs(t.leaf_y[a] - t.leaf_y[b])) <= 1) ? 1 : 0;
            for (int nu = L; nu >= 1; nu--) {
                int sh = 2 * (L - nu);
                cover += (int)pairs[nu].count((long)(a >> sh) * t.lv[nu].nbox + (b >> sh));
            }
            if (cover != 1) bad++;
        }
    return bad;
}

}  // namespace dafmm
