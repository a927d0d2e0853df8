// spc_sort_fitness_static: the fitness sort (S4) for callers that cannot allocate GPU memory.
//
// Some callers of this library must not call cudaMalloc: code that runs under another
// framework's fixed memory budget or pool and may not grow it, latency-critical threads that
// cannot afford cudaMalloc's implicit device-wide synchronisation, and embedded uses where all
// device memory is reserved up front.  spc_sort_fitness needs a context, and a context
// allocates its workspace.  This entry point needs neither: the caller passes the input and
// the output in device memory, and every temporary lives in one file-scope device array,
// g_static_scratch, which is part of the library's module image.  Every GPU that loads the
// library holds that array (kStaticScratchBytes) until the process exits.
//
// Set-up: the first call on a device, with that device current, looks up the array's device
// address with cudaGetSymbolAddress (in host code the array's name is only a host-side stand-in,
// not a device address) and caches it per device; later calls reuse it.  Make that first call
// before any stream capture.
//
// Every call shares the one array, and it keeps the previous call's contents.  No part of it
// needs to start at zero: each kernel writes every scratch element it later reads (keys,
// histograms, scan partials).  Calls whose work can run at the same time on the GPU (different
// streams without ordering between them) race on the array and give wrong results; order them
// on one stream or with events.
#include <mutex>

#include "spc_internal.cuh"

namespace {

// largest m the static scratch can sort
constexpr int64_t kStaticMaxEdges = int64_t(1) << 20;

// keys + alternate keys (uint64), alternate values (uint32), radix histograms, scan partials
constexpr size_t kStaticScratchBytes = size_t(22) << 20;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_dev[kMaxDevices] = {};

// device address of g_static_scratch on the current device (looked up once per device)
spc_status static_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        spc::set_last_cuda_error(e, "cudaGetDevice", __FILE__, __LINE__);
        return SPC_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return SPC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            spc::set_last_cuda_error(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
            return SPC_ERR_CUDA;
        }
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return SPC_OK;
}

// device (or managed) memory that the current device's kernels can read: memory of another
// GPU is refused, since the kernels would read it without peer access
bool on_device(const void* p) {
    cudaPointerAttributes a;
    int dev = -1;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// keys = score bits (uint32 scores widened), values = edge ids
template <class KT>
__global__ void k_static_prep(int64_t m, const KT* __restrict__ f, uint64_t* __restrict__ key,
                              uint32_t* __restrict__ val) {
    spc::pdl_wait();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        key[e] = (uint64_t)f[e];
        val[e] = (uint32_t)e;
    }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" spc_status spc_sort_fitness_static(int64_t m, const void* f, spc_dtype ftype,
                                              int32_t* order_out, void* stream) {
    if (m < 0 || (ftype != SPC_F32 && ftype != SPC_F64)) return SPC_ERR_INVALID_ARG;
    if (m > kStaticMaxEdges) return SPC_ERR_TOO_LARGE;
    if (m == 0) return SPC_OK;
    if (!f || !order_out || !on_device(f) || !on_device(order_out)) return SPC_ERR_INVALID_ARG;
    void* base = nullptr;
    spc_status st = static_scratch(&base);
    if (st != SPC_OK) return st;
    // carve the array: keys | keys_alt | vals_alt | hist | scan partials
    unsigned char* p = static_cast<unsigned char*>(base);
    size_t off = 0;
    uint64_t* keys = reinterpret_cast<uint64_t*>(p + off);
    off += align256((size_t)kStaticMaxEdges * 8);
    uint64_t* keys_alt = reinterpret_cast<uint64_t*>(p + off);
    off += align256((size_t)kStaticMaxEdges * 8);
    uint32_t* vals_alt = reinterpret_cast<uint32_t*>(p + off);
    off += align256((size_t)kStaticMaxEdges * 4);
    const int64_t hist_elems = spc::radix_raw_hist_elems(kStaticMaxEdges);
    int32_t* hist = reinterpret_cast<int32_t*>(p + off);
    off += align256((size_t)hist_elems * 4);
    int32_t* scan_tmp = reinterpret_cast<int32_t*>(p + off);
    off += align256((size_t)spc::scan_raw_tmp_elems(hist_elems) * 4);
    if (off > kStaticScratchBytes) return SPC_ERR_TOO_LARGE;  // layout guard

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t* vals = reinterpret_cast<uint32_t*>(order_out);
    const int blocks = (int)((m + 255) / 256 < 4096 ? (m + 255) / 256 : 4096);
    if (ftype == SPC_F64)
        k_static_prep<uint64_t><<<blocks, 256, 0, s>>>(m, static_cast<const uint64_t*>(f), keys, vals);
    else
        k_static_prep<uint32_t><<<blocks, 256, 0, s>>>(m, static_cast<const uint32_t*>(f), keys, vals);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = spc::radix_sort_u64_raw(s, keys, vals, keys_alt, vals_alt, m,
                                    ftype == SPC_F64 ? 63 : 31, hist, scan_tmp);
    if (e != cudaSuccess) {
        spc::set_last_cuda_error(e, "spc_sort_fitness_static", __FILE__, __LINE__);
        return SPC_ERR_CUDA;
    }
    return SPC_OK;
}
