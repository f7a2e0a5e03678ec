// Field readback that allocates no device memory.
//
// lbm_get_rho_u stages every chunk of results in a buffer it obtains from the
// lattice's allocator for the duration of the call.  Some callers cannot
// allocate at that point: a simulation sized to fill the GPU (16-bit 1024^3
// lattices leave little room) would see the allocation fail, and in
// processes where another framework owns the device memory pool, or where a
// blocking cudaMalloc would stall other streams in the middle of a time loop,
// allocating is not acceptable.  lbm_get_rho_u_static runs the same
// field-probe kernel but stages through the fixed array below.  Its device
// address is looked up when the first lattice on a device is created (which
// also makes the runtime place the array there), so a readback in the middle
// of a run takes no memory.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "lbm.h"
#include "lbm_handle.h"

namespace {

constexpr size_t kStaticDoubles = size_t(1) << 20;   // 8 MiB per device

// Shared by every call on a device; each chunk is fully written before it is read.
static __device__ __align__(256) double g_rho_u_stage[kStaticDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_stage_mutex;
double* g_stage_addr[kMaxDevices] = {};   // device address of g_rho_u_stage, per device
bool g_stage_tried[kMaxDevices] = {};     // look-up done (g_stage_addr stays NULL if it failed)

template <class R>
lbm_status fields_static(lbm_handle* h, const Relax<R>& k, double* stage, double* dst[4]) {
    const size_t plane = (size_t)h->p.nx * h->p.ny;
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(kStaticDoubles / (4 * plane), (size_t)h->p.nz));
    for (int z0 = 0; z0 < h->p.nz; z0 += chunk) {
        const int z1 = std::min(h->p.nz, z0 + chunk);
        lbm::ProbeArgs<R> pa{};
        pa.a = h->args(k, h->aa() ? 0 : h->cur);
        pa.z0 = z0;
        pa.z1 = z1;
        pa.out = stage;
        pa.partial = h->partial;
        const size_t count = plane * (size_t)(z1 - z0);
        Launch L;
        L.block = dim3(256);
        L.grid = dim3((unsigned)std::min<size_t>((count + 255) / 256, 152 * 32));
        L.stream = h->stream;
        if (h->cuda(h->ks->probe[h->layout_now()](&pa, lbm::PROBE_FIELDS, L), "probe kernel")) return LBM_ERR_CUDA;
        for (int c = 0; c < 4; ++c)
            if (dst[c] && h->cuda(cudaMemcpyAsync(dst[c] + plane * z0, stage + c * count, count * sizeof(double),
                                                  cudaMemcpyDeviceToHost, h->stream), "fields download"))
                return LBM_ERR_CUDA;
        // the next chunk reuses the array
        if (h->cuda(cudaStreamSynchronize(h->stream), "sync")) return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

}  // namespace

// In host code the array's name only stands for the symbol, so its device
// address is asked for once per device, with that device current.
double* lbm_internal_static_stage() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_stage_mutex);
    if (!g_stage_tried[dev]) {
        g_stage_tried[dev] = true;
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_rho_u_stage) == cudaSuccess) g_stage_addr[dev] = static_cast<double*>(p);
        else cudaGetLastError();   // not sticky: the lattice itself is unaffected
    }
    return g_stage_addr[dev];
}

extern "C" lbm_status lbm_get_rho_u_static(lbm_handle* h, double* rho, double* ux, double* uy, double* uz) {
    if (!h) return LBM_ERR_ARG;
    if (h->sticky != LBM_OK) return LBM_ERR_STATE;
    const size_t plane = (size_t)h->p.nx * h->p.ny;
    if (4 * plane > kStaticDoubles)
        return h->fail(LBM_ERR_UNSUPPORTED,
                       "lbm_get_rho_u_static: an xy-plane needs " + std::to_string(4 * plane) +
                           " doubles of staging, the static buffer holds " + std::to_string(kStaticDoubles) +
                           " (nx*ny must not exceed 262144); use lbm_get_rho_u");
    if (!h->static_stage)
        return h->fail(LBM_ERR_UNSUPPORTED,
                       "lbm_get_rho_u_static: the static staging array could not be placed on this device "
                       "when the lattice was created; use lbm_get_rho_u");
    double* dst[4] = {rho, ux, uy, uz};
    const lbm_status st = h->fp64() ? fields_static(h, h->kd, h->static_stage, dst)
                                    : fields_static(h, h->kf, h->static_stage, dst);
    return st == LBM_OK ? lbm_internal_check_status(h) : st;
}
