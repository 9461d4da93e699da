// noalloc.cu -- nmodl_cur_noalloc: the current update (nrn_cur) for callers
// that cannot allocate device memory.
//
// The regular path keeps a per-mechanism chunk table (segment-aligned warp
// chunks of the node_index-sorted reduction) and a parameter descriptor in
// memory that nmodl_mech_create allocates.  Some callers cannot do that:
// code running inside another framework's memory pool or a host that forbids
// cudaMalloc after start-up, or a step function that must not touch the
// allocator at all.  This entry point instead keeps that scratch in one
// fixed, file-scope device array (kScratchBytes per GPU that loads the
// library, held until the process exits) and allocates nothing.
#include <mutex>

#include "kernels.cuh"

namespace nmodl {

// internal helper defined in api.cu: parameter block -> device descriptor
int build_desc_for(int type, const double* params, int64_t n_params, MechD* md,
                   Kin9D* kd, int* n_states);

namespace {

constexpr size_t kScratchBytes = 1u << 20;  // 1 MiB per device
constexpr size_t kFlagsOff = 0;             // int32 flags: [0] validation, [1] non-finite
constexpr size_t kDescOff = 256;            // MechD or Kin9D
constexpr size_t kChunkOff = 1280;          // int32 chunk table
constexpr int64_t kMaxChunks = (int64_t)((kScratchBytes - kChunkOff) / 4) - 1;
constexpr int64_t kMaxInstances = 8000000;  // <= 32 * kMaxChunks
static_assert(kMaxInstances <= 32 * kMaxChunks, "scratch too small");
static_assert(sizeof(MechD) <= kChunkOff - kDescOff, "descriptor slot");
static_assert(sizeof(Kin9D) <= kChunkOff - kDescOff, "descriptor slot");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_ptr[kMaxDevices] = {};

}  // namespace

static __device__ __align__(256) unsigned char g_cur_scratch[kScratchBytes];

// Device address of g_cur_scratch on the current device; resolved once per
// device (the host-side name of the array is not a device address).
static int scratch_ptr(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return NMODL_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_cur_scratch);
        if (e != cudaSuccess || !p) return NMODL_ERR_CUDA;
        g_ptr[device] = (unsigned char*)p;
    }
    *out = g_ptr[device];
    return NMODL_OK;
}

}  // namespace nmodl

using namespace nmodl;

extern "C" NMODL_API int64_t nmodl_cur_noalloc_max_instances(void) { return kMaxInstances; }

extern "C" NMODL_API int nmodl_cur_noalloc(int device, void* cuda_stream, int type,
                                           int64_t n_instances, const int32_t* node_index,
                                           int64_t n_nodes, const double* params,
                                           int64_t n_params, const double* states,
                                           int64_t stride, const double* v, double* rhs,
                                           double* d) {
    if (n_instances < 0 || n_nodes < 0 || stride < n_instances || !params)
        return NMODL_ERR_ARG;
    if (n_instances > kMaxInstances) return NMODL_ERR_TOO_LARGE;
    if (type != NMODL_HH && type != NMODL_CNEXP && type != NMODL_KIN9)
        return NMODL_ERR_UNSUPPORTED;
    MechD md{};
    Kin9D kd{};
    int n_states = 0;
    int rc = build_desc_for(type, params, n_params, &md, &kd, &n_states);
    if (rc) return rc;
    if (n_instances == 0) return NMODL_OK;
    if (!node_index || (n_states > 0 && !states) || !v || !rhs || !d) return NMODL_ERR_ARG;

    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return NMODL_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned char* base = nullptr;
    rc = scratch_ptr(device, &base);
    if (rc == NMODL_OK) {
        int32_t* flags = (int32_t*)(base + kFlagsOff);
        void* desc = base + kDescOff;
        int32_t* chunk = (int32_t*)(base + kChunkOff);
        const int64_t n_chunks = (n_instances + 31) / 32;
        cudaError_t e = cudaMemsetAsync(flags, 0, 2 * sizeof(int32_t), s);
        if (e == cudaSuccess)
            e = (type == NMODL_KIN9)
                    ? cudaMemcpyAsync(desc, &kd, sizeof(kd), cudaMemcpyHostToDevice, s)
                    : cudaMemcpyAsync(desc, &md, sizeof(md), cudaMemcpyHostToDevice, s);
        // node_index must be sorted and in range before the reduction reads
        // v[node]: validate first and stop with an error otherwise.
        int32_t hflags = 0;
        if (e == cudaSuccess) {
            launch_validate_index(node_index, n_instances, n_nodes, flags, s);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = NMODL_ERR_CUDA;
        } else if (hflags & 2) {
            rc = NMODL_ERR_RANGE;
        } else if (hflags & 1) {
            rc = NMODL_ERR_UNSORTED;
        } else {
            // A non-finite rhs or d of this call is latched in flags[1] and
            // read back once the reduction has finished, so the call reports
            // it as nmodl_cur's context would (there is no context here).
            launch_chunk_starts(node_index, n_instances, n_chunks, chunk, s);
            launch_cur_seg(type == NMODL_KIN9 ? NMODL_KIN9 : NMODL_CNEXP, desc, n_chunks,
                           chunk, node_index, v, states, stride, rhs, d, nullptr, nullptr,
                           flags + 1, s);
            int32_t hbad = 0;
            e = cudaGetLastError();
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&hbad, flags + 1, sizeof(hbad), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) rc = NMODL_ERR_CUDA;
            else if (hbad) rc = NMODL_ERR_NONFINITE;
        }
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return rc;
}
