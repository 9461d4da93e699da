// k_common.cu -- bookkeeping kernels: node_index validation, the
// segment-aligned warp chunk table of the current reduction, tile bounds of
// the fused step, and the diagonal voltage update of the generic step.
#include "kernels.cuh"

namespace nmodl {

// flags[0] |= 1 if some node_index[j] < node_index[j-1] (unsorted),
// flags[0] |= 2 if some value lies outside [0, n_nodes).
__global__ void k_validate_index(const int32_t* __restrict__ ni, int64_t n,
                                 int64_t n_nodes, int32_t* flags) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = ni[j];
        int f = 0;
        if (x < 0 || (int64_t)x >= n_nodes) f |= 2;
        if (j > 0 && ni[j - 1] > x) f |= 1;
        if (f) atomicOr(flags, f);
    }
}

// first index in [lo, hi) with ni[index] > key (ni sorted)
__device__ __forceinline__ int64_t upper_bound_i32(const int32_t* ni, int64_t lo,
                                                   int64_t hi, int32_t key) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (ni[mid] <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// first index in [lo, hi) with ni[index] >= key
__device__ __forceinline__ int64_t lower_bound_i32(const int32_t* ni, int64_t lo,
                                                   int64_t hi, int64_t key) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)ni[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// chunk[c] = first segment head at or after 32c (n if none), c in [0, n_chunks]
__global__ void k_chunk_starts(const int32_t* __restrict__ ni, int64_t n,
                               int64_t n_chunks, int32_t* chunk) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c > n_chunks) return;
    const int64_t j = c * 32;
    int64_t out;
    if (j >= n) out = n;
    else if (j == 0 || ni[j] != ni[j - 1]) out = j;
    else out = upper_bound_i32(ni, j, n, ni[j]);
    chunk[c] = (int32_t)out;
}

// out[k] = first instance whose node is >= nodes[k]
__global__ void k_tile_bounds(const int32_t* __restrict__ ni, int64_t n,
                              const int64_t* __restrict__ nodes, int64_t n_bounds,
                              int32_t* out) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n_bounds) return;
    out[k] = (int32_t)lower_bound_i32(ni, 0, n, nodes[k]);
}

// d += 1e-3 cm/dt; v += rhs/d (unless clamped; the quotient within one ulp
// by the two-FP64-instruction division of the gate updates)
__global__ void k_vupdate(int64_t n_nodes, double* v, const double* __restrict__ rhs,
                          double* d, double cmdt, int clamp, int32_t* err) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_nodes;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double dd = d[k] + cmdt;
        d[k] = dd;
        if (!clamp) {
            const double vn = v[k] + ddiv_fast(rhs[k], dd);
            if (!finite_int(vn)) latch_error(err, NMODL_ERR_NONFINITE);
            v[k] = vn;
        }
    }
}

static int grid_1d(int64_t n, int block) {
    int64_t b = (n + block - 1) / block;
    if (b > 148 * 32) b = 148 * 32;
    return (int)(b < 1 ? 1 : b);
}

void launch_validate_index(const int32_t* ni, int64_t n, int64_t n_nodes,
                           int32_t* flags, cudaStream_t s) {
    if (n == 0) return;
    k_validate_index<<<grid_1d(n, 256), 256, 0, s>>>(ni, n, n_nodes, flags);
}

void launch_chunk_starts(const int32_t* ni, int64_t n, int64_t n_chunks,
                         int32_t* chunk, cudaStream_t s) {
    const int64_t m = n_chunks + 1;
    k_chunk_starts<<<(int)((m + 255) / 256), 256, 0, s>>>(ni, n, n_chunks, chunk);
}

void launch_tile_bounds(const int32_t* ni, int64_t n, const int64_t* nodes,
                        int64_t n_bounds, int32_t* out, cudaStream_t s) {
    if (n_bounds == 0) return;
    k_tile_bounds<<<(int)((n_bounds + 255) / 256), 256, 0, s>>>(ni, n, nodes, n_bounds, out);
}

void launch_vupdate(int64_t n_nodes, double* v, const double* rhs, double* d,
                    double cmdt, int clamp, int32_t* err, cudaStream_t s) {
    if (n_nodes == 0) return;
    k_vupdate<<<grid_1d(n_nodes, 256), 256, 0, s>>>(n_nodes, v, rhs, d, cmdt, clamp, err);
}

}  // namespace nmodl
