// Internal declarations of the DAFMM library (not part of the C-ABI).
#pragma once

#include <complex>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "dafmm.h"

namespace dafmm {

using cd = std::complex<double>;

// Exception carrying a DAFMM_E* status; converted to a return code at the C-ABI.
struct Status : std::runtime_error {
    int code;
    Status(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

[[noreturn]] inline void fail(int code, const std::string& msg) { throw Status(code, msg); }

void set_last_error(int code, const std::string& msg);

// ---------------------------------------------------------------- tree ----

// One level of the uniform quadtree.  A "slot" is a box at a low-frequency
// level and a (box, cone) pair at a high-frequency level: slot = box * nc + cone.
struct Level {
    int nu = 0;        // level index (0 = root)
    int nside = 0;     // boxes per side
    int nbox = 0;      // nside^2, boxes in Morton order
    int nc = 1;        // cones per box (1 when low frequency)
    double w = 0;      // box half-width
    bool hf = false;   // high-frequency regime: (kappa w)^2 > T
    // interaction lists per slot: slots of the same level (Table 1)
    std::vector<int> il_ptr, il_idx;
    // slot takes part in the far field (own list non-empty, or a related
    // parent slot does)
    std::vector<char> active;
    int nslot() const { return nbox * nc; }
};

struct Tree {
    dafmm_params prm{};
    int n_side = 0, p = 4, nb = 0, L = 0, top = 0;
    long N = 0;
    double x0 = 0, x1 = 0, beta = 0;  // beta: leaf half-width
    std::vector<Level> lv;            // 0..L
    std::vector<int> leaf_x, leaf_y;  // leaf coordinates by Morton index
};

void morton_decode(long m, int* x, int* y);
long morton_encode(int x, int y);

// Build the tree, lists and cones; throws Status on bad input.
Tree* make_tree(const dafmm_params& prm, int n_side, double x0, double x1);

// Leaf pairs not covered exactly once, plus unmatched directional entries.
long check_tree(const Tree& t);

// Slots of level nu+1 related to slot s of level nu: the children used by
// M2M / reached by L2L (Section 4.2.1, four cases).
void child_slots(const Tree& t, int nu, int s, std::vector<int>& out);

// Chebyshev nodes (ascending, first kind) used by the library.
void cheb_nodes(int p, double* z);

// ------------------------------------------------------------ operators ----

// Block-sparse operator: for each output row r, y[r] (+)= sum_e M_e x[col_e].
// Block e is rout[r] x rin[e] complex at its realised ranks, stored
// column-major (output index fastest) with column stride ld[r] = rout[r]
// rounded up to even, at offset moff[e] of mats; a row's blocks follow each
// other, so the row is one ld x (sum of rin) matrix starting at an even offset.
struct BsrHost {
    int nrows = 0;
    int Rout = 0, Rin = 0;  // largest rout / rin (strides of the coefficient buffers)
    std::vector<int> rowptr, col;
    std::vector<int> rout;  // per row
    std::vector<int> ld;    // per row: column stride (rout rounded up to even)
    std::vector<int> rin;   // per entry
    std::vector<long> moff; // per entry, in complex elements
    std::vector<cd> mats;
    long nnz() const { return (long)col.size(); }
    // fill ld, moff and size mats from rowptr, rout and rin
    void layout()
    {
        moff.assign(col.size(), 0);
        ld.assign(nrows, 0);
        long off = 0;
        for (int r = 0; r < nrows; r++) {
            ld[r] = rout[r] + (rout[r] & 1);
            for (int e = rowptr[r]; e < rowptr[r + 1]; e++) {
                moff[e] = off;
                off += (long)ld[r] * rin[e];
            }
        }
        mats.assign((size_t)off, cd(0));
    }
};

struct BsrDev {
    int nrows = 0, Rout = 0, Rin = 0;
    long nnz = 0, nelem = 0;
    int* rout = nullptr;
    int* col = nullptr;
    int* rin = nullptr;
    long* moff = nullptr;
    int* rowptr = nullptr;
    void* m32 = nullptr;  // float2 blocks
    void* mdf = nullptr;  // float4 blocks {re hi, im hi, re lo, im lo}: complex128 as float pairs
};

// Everything the matvec needs, produced on the host by the NCA setup.
struct LevelOpsHost {
    int Ri = 0, Ro = 0;       // padded incoming / outgoing ranks
    std::vector<int> ri, ro;  // realised ranks per slot
    BsrHost up;    // rows: slots of nu, cols: slots of nu+1 (leaf: leaves of v)
    BsrHost m2l;   // rows: slots of nu, cols: slots of nu
    BsrHost down;  // rows: slots of nu+1, cols: slots of nu (leaf: L2P, rows leaves)
};

struct OpsHost {
    std::vector<LevelOpsHost> lv;  // 0..L; only top..L used
    std::vector<cd> near;          // 9 x 16 x 16 near-field blocks, offset (dx,dy) -> (dy+1)*3+(dx+1)
    double t_nca = 0;
};

// Host copy of the offset table K(offset, i', j') built on the device.
struct EntryTable {
    int nb = 0, p = 4, n2 = 16;
    std::vector<cd> tab;  // ((dy + nb-1) * (2nb-1) + (dx + nb-1)) * 256 + i' * 16 + j'
    const std::vector<int>* lx = nullptr;
    const std::vector<int>* ly = nullptr;
    inline cd operator()(long i, long j) const {
        long bi = i >> 4, bj = j >> 4;
        int dx = (*lx)[bi] - (*lx)[bj] + nb - 1;
        int dy = (*ly)[bi] - (*ly)[bj] + nb - 1;
        return tab[(((long)dy * (2 * nb - 1) + dx) * 16 + (i & 15)) * 16 + (j & 15)];
    }
};

void build_nca(const Tree& t, const EntryTable& K, OpsHost& ops);

// Build the offset table on the device (entries.cu); returns seconds spent.
double build_entry_table(const Tree& t, EntryTable& out, void* stream);

}  // namespace dafmm
