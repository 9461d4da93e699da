// k_cable.cu -- cable coupling: the per-cell tree (Hines) solve that
// replaces the diagonal voltage update when compartments form cells.
//
// For each non-root node i with parent p (p < i inside a contiguous cell),
// axial conductances ga[i] (per unit area of i) and gb[i] (per unit area of
// p) add rhs[i] += ga (v[p] - v[i]), rhs[p] += gb (v[i] - v[p]),
// d[i] += ga, d[p] += gb, and the off-diagonals M[i][p] = -ga, M[p][i] = -gb.
// Because every parent precedes its children, Gaussian elimination from the
// last node to the root creates no fill (Hines 1984):
//   leaf -> root:  f = gb[i]/d[i];  d[p] -= f ga[i];  rhs[p] += f rhs[i]
//   root:          dv = rhs/d
//   root -> leaf:  dv[i] = (rhs[i] + ga[i] dv[p]) / d[i]
// and v += dv.  One thread owns one cell; the eliminated system lives in
// the cable's scratch arrays so that rhs and d keep the assembled values.
#include "kernels.cuh"

namespace nmodl {

__global__ void k_cable_solve(int64_t n_cells, const int64_t* __restrict__ cell_off,
                              const int32_t* __restrict__ parent,
                              const double* __restrict__ ga, const double* __restrict__ gb,
                              double cmdt, double* v, double* rhs, double* d, double* d2,
                              double* r2, int clamp, int32_t* err) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const int64_t a = cell_off[c], b = cell_off[c + 1];
    for (int64_t i = a; i < b; ++i) {
        d2[i] = d[i] + cmdt;
        r2[i] = rhs[i];
    }
    for (int64_t i = a + 1; i < b; ++i) {
        const int64_t p = parent[i];
        const double dv = v[i] - v[p];
        r2[i] -= ga[i] * dv;
        r2[p] += gb[i] * dv;
        d2[i] += ga[i];
        d2[p] += gb[i];
    }
    for (int64_t i = a; i < b; ++i) {
        d[i] = d2[i];
        rhs[i] = r2[i];
    }
    if (clamp) return;  // v held: the assembled system is reported, not solved
    for (int64_t i = b - 1; i > a; --i) {
        const int64_t p = parent[i];
        const double f = gb[i] / d2[i];
        d2[p] -= f * ga[i];
        r2[p] += f * r2[i];
    }
    r2[a] = r2[a] / d2[a];
    for (int64_t i = a + 1; i < b; ++i) r2[i] = (r2[i] + ga[i] * r2[parent[i]]) / d2[i];
    for (int64_t i = a; i < b; ++i) {
        const double vn = v[i] + r2[i];
        if (!finite_int(vn)) latch_error(err, NMODL_ERR_NONFINITE);
        v[i] = vn;
    }
}

void launch_cable_solve(int64_t n_cells, const int64_t* cell_off, const int32_t* parent,
                        const double* ga, const double* gb, double cmdt, double* v,
                        double* rhs, double* d, double* d2, double* r2, int clamp,
                        int32_t* err, cudaStream_t s) {
    if (n_cells == 0) return;
    const int block = 64;
    k_cable_solve<<<(int)((n_cells + block - 1) / block), block, 0, s>>>(
        n_cells, cell_off, parent, ga, gb, cmdt, v, rhs, d, d2, r2, clamp, err);
}

}  // namespace nmodl
