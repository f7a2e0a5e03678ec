// Host implementation of the C ABI declared in include/lbm.h.
// Validates arguments, owns device memory through the caller's allocator,
// moves data in bounded chunks and launches the kernels of lbm_kernels.cuh.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_handle.h"
#include "lbm_kernels.cuh"
#include "lbm_registry.h"

using namespace lbm;

namespace lbm {
KernelSet& kernel_set(int velset, int collision, int storage, int arith) {
    static KernelSet table[3][3][10][2];
    return table[velset][collision][storage][arith];
}
}  // namespace lbm

namespace {

constexpr size_t kScratchDoubles = size_t(16) << 20;   // 128 MB staging
constexpr int kReduceBlocks = 152 * 8;

int velset_q(int v) { return v == LBM_D2Q9 ? 9 : (v == LBM_D3Q19 ? 19 : 27); }
int storage_bytes(int s) { return s == LBM_FP64 ? 8 : (s == LBM_FP32 ? 4 : 2); }

void* default_alloc(size_t bytes, void*) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
void default_release(void* p, void*) { cudaFree(p); }

}  // namespace

namespace {

template <class R> void make_relax(const lbm_params& p, Relax<R>& k) {
    k.om = (R)(1.0 / p.tau);
    k.c1 = (R)1 - k.om;
    k.omp = k.om;
    k.omm = (R)(1.0 / (p.trt_lambda / (p.tau - 0.5) + 0.5));
    k.cSp = (R)1 - (R)0.5 * k.omp;
    k.cSm = (R)1 - (R)0.5 * k.omm;
    k.omph = (R)0.5 * k.omp;
    k.ommh = (R)0.5 * k.omm;
    k.cSph = (R)0.5 * k.cSp;
    k.cSmh = (R)0.5 * k.cSm;
    k.cs = (R)(1.0 / std::sqrt(3.0));
    for (int a = 0; a < 3; ++a) k.F[a] = (R)p.force[a];
    k.force = (p.force[0] != 0.0 || p.force[1] != 0.0 || p.force[2] != 0.0) ? 1 : 0;
    // force components that keep a nonzero numerator j_a + F_a/2 of the
    // 16-bit formats at or above 2^-100 in magnitude (numerators_ok)
    k.xsafe = 1;
    for (int a = 0; a < 3; ++a) {
        const double fa = std::fabs((double)k.F[a]);
        if (fa != 0.0 && (fa < 0x1p-76 || fa > 0x1p90)) k.xsafe = 0;
    }
    k.sh = p.no_ddf_shifting ? (R)0 : (R)1;
    if (p.collision == LBM_MRT) {   // D3Q19 rates of d'Humieres et al. (2002); shear and conserved: omega
        const double om = 1.0 / p.tau;
        const double s[19] = {om, 1.19, 1.4, om, 1.2, om, 1.2, om, 1.2, om, 1.4, om, 1.4, om, om, om, 1.98, 1.98, 1.98};
        for (int kk = 0; kk < 19; ++kk) {
            double norm = 0.0;
            for (int i = 0; i < 19; ++i) {
                const double e = (double)mrt_m<D3Q19>(kk, i);
                norm += e * e;
            }
            k.mrt_r[kk] = (R)(s[kk] / norm);
            k.mrt_p[kk] = (R)((1.0 - 0.5 * s[kk]) / norm);
        }
    }
}

bool want_chunked(const lbm_handle* h);
lbm_status ensure_layout(lbm_handle* h);
lbm_status zero_solid(lbm_handle* h);

lbm_status check_handle(lbm_handle* h) {
    if (!h) return LBM_ERR_ARG;
    if (h->sticky != LBM_OK) return LBM_ERR_STATE;
    return LBM_OK;
}

// Staging buffer for host transfers, held only for the duration of one call
// (an ensemble of hundreds of lattices would otherwise hold hundreds of them).
struct Staging {
    lbm_handle* h;
    explicit Staging(lbm_handle* hh) : h(hh) {
        h->scratch = (double*)h->alloc(h->scratch_doubles * sizeof(double));
    }
    ~Staging() {
        if (h->scratch) {
            cudaStreamSynchronize(h->stream);
            h->release((void*&)h->scratch, h->scratch_doubles * sizeof(double));
        }
    }
    bool ok() const { return h->scratch != nullptr; }
};

// Device buffer from the lattice's allocator, released (after the stream has
// drained) when the call returns.
struct TempBuffer {
    lbm_handle* h;
    size_t bytes;
    void* p = nullptr;
    TempBuffer(lbm_handle* hh, size_t b) : h(hh), bytes(b) { p = bytes ? h->alloc(bytes) : nullptr; }
    ~TempBuffer() {
        if (p) {
            cudaStreamSynchronize(h->stream);
            h->release(p, bytes);
        }
    }
};

constexpr size_t kListChunk = size_t(1) << 20;   // cells per probe / scatter launch

lbm_status check_cell_list(lbm_handle* h, int64_t count, const int64_t* cells) {
    if (count < 0) return h->fail(LBM_ERR_ARG, "negative cell count");
    if (count > 0 && !cells) return h->fail(LBM_ERR_ARG, "cells is NULL");
    for (int64_t k = 0; k < count; ++k)
        if (cells[k] < 0 || cells[k] >= (int64_t)h->N)
            return h->fail(LBM_ERR_ARG, "cell index " + std::to_string(cells[k]) + " at position " + std::to_string(k) +
                                            " is outside [0, " + std::to_string(h->N) + ")");
    return LBM_OK;
}

// reads the device status word (call after a stream synchronisation)
lbm_status check_status(lbm_handle* h) {
    int st = 0;
    if (h->cuda(cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost), "status read")) return LBM_ERR_CUDA;
    if (st) {
        h->sticky = LBM_ERR_TIMEOUT;
        h->err = "a kernel gave up waiting for its staged copies";
        return LBM_ERR_TIMEOUT;
    }
    return LBM_OK;
}

}  // namespace

extern "C" const char* lbm_status_string(lbm_status s) {
    switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_OOM: return "out of device memory";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_UNSUPPORTED: return "unsupported combination";
    case LBM_ERR_DIVERGED: return "simulation diverged";
    case LBM_ERR_TIMEOUT: return "timeout";
    case LBM_ERR_STATE: return "handle in error state";
    }
    return "unknown status";
}

extern "C" const char* lbm_last_error(const lbm_handle* h) { return h ? h->err.c_str() : "null handle"; }

extern "C" lbm_status lbm_create(const lbm_params* params, const lbm_allocator* allocator, void* cuda_stream,
                      lbm_handle** out) {
    if (!params || !out) return LBM_ERR_ARG;
    *out = nullptr;
    const lbm_params& p = *params;
    if (p.nx < 1 || p.ny < 1 || p.nz < 1) return LBM_ERR_ARG;
    if (p.velset < LBM_D2Q9 || p.velset > LBM_D3Q27) return LBM_ERR_ARG;
    if (p.velset == LBM_D2Q9 && p.nz != 1) return LBM_ERR_ARG;
    if (p.collision != LBM_SRT && p.collision != LBM_TRT && p.collision != LBM_MRT) return LBM_ERR_ARG;
    if (p.collision == LBM_MRT && p.velset != LBM_D3Q19) return LBM_ERR_UNSUPPORTED;
    if (p.storage < LBM_FP64 || p.storage > LBM_P16_1) return LBM_ERR_ARG;
    if (p.arith != LBM_ARITH_FP32 && p.arith != LBM_ARITH_FP64) return LBM_ERR_ARG;
    if (p.scheme != LBM_STREAM_AB && p.scheme != LBM_STREAM_AA && p.scheme != LBM_STREAM_AUTO) return LBM_ERR_ARG;
    if (!(p.tau > 0.5) || !std::isfinite(p.tau)) return LBM_ERR_ARG;
    if (p.collision == LBM_TRT && !(p.trt_lambda > 0.0 && std::isfinite(p.trt_lambda))) return LBM_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(p.force[a])) return LBM_ERR_ARG;
    const size_t N = (size_t)p.nx * p.ny * p.nz;
    if (N > 0x7FFFFFFFull) return LBM_ERR_UNSUPPORTED;
    if (p.arith == LBM_ARITH_FP64 && p.storage != LBM_FP64 && p.storage != LBM_FP32)
        return LBM_ERR_UNSUPPORTED;

    lbm_handle* h = new lbm_handle;
    h->p = p;
    if (p.scheme == LBM_STREAM_AUTO) {   // A-B when both copies fit with a 10% margin
        h->scheme_auto = true;
        size_t free_b = 0, total_b = 0;
        const double need = 2.0 * (double)velset_q(p.velset) * (double)N * storage_bytes(p.storage);
        const bool fits = cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && need * 1.1 < (double)free_b;
        if (!fits) cudaGetLastError();
        h->p.scheme = fits ? LBM_STREAM_AB : LBM_STREAM_AA;
    }
    if (p.velset == LBM_D2Q9) h->p.force[2] = 0.0;
    if (p.collision == LBM_SRT) h->p.trt_lambda = p.trt_lambda > 0 ? p.trt_lambda : 0.1875;
    h->q = velset_q(p.velset);
    h->N = N;
    h->sb = storage_bytes(p.storage);
    if (allocator && allocator->alloc && allocator->release) h->al = *allocator;
    else h->al = lbm_allocator{default_alloc, default_release, nullptr};
    h->stream = (cudaStream_t)cuda_stream;
    h->ks = &kernel_set(p.velset, p.collision, p.storage, p.arith);
    if (!h->ks->present) {
        delete h;
        return LBM_ERR_UNSUPPORTED;
    }
    make_relax(h->p, h->kf);
    make_relax(h->p, h->kd);

    const size_t fbytes = h->fbytes();
    const int copies = h->aa() ? 1 : 2;
    for (int c = 0; c < copies; ++c) {
        h->f[c] = h->alloc(fbytes);
        if (!h->f[c]) { lbm_destroy(h); return LBM_ERR_OOM; }
    }
    h->scratch_doubles = std::max(kScratchDoubles, (size_t)h->plane() * std::max(h->q, 4));
    h->scratch_doubles = std::min(h->scratch_doubles, (size_t)std::max(h->q, 4) * N);
    h->partial = (double*)h->alloc((2 * kReduceBlocks + 2) * sizeof(double) + 256);
    if (!h->partial) { lbm_destroy(h); return LBM_ERR_OOM; }
    h->status = (int*)(h->partial + 2 * kReduceBlocks + 2);
    if (h->cuda(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream), "memset")) {
        lbm_destroy(h);
        return LBM_ERR_CUDA;
    }
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (h->num_sms <= 0) h->num_sms = 1;
    }
    // lbm_get_rho_u_static's array is placed now, while the device has room
    h->static_stage = lbm_internal_static_stage();
    for (int c = 0; c < copies; ++c)
        if (h->cuda(cudaMemsetAsync(h->f[c], 0, fbytes, h->stream), "memset") != LBM_OK) {
            lbm_destroy(h);
            return LBM_ERR_CUDA;
        }
    if (p.no_ddf_shifting) {   // zero populations are rest only when shifted
        const lbm_status st = lbm_set_rho_u(h, nullptr, nullptr, nullptr, nullptr);
        if (st != LBM_OK) {
            lbm_destroy(h);
            return st;
        }
    }
    *out = h;
    return LBM_OK;
}

extern "C" lbm_status lbm_destroy(lbm_handle* h) {
    if (!h) return LBM_OK;
    cudaStreamSynchronize(h->stream);
    for (auto& row : h->graph)
        for (auto& g : row)
            if (g) cudaGraphExecDestroy(g);
    if (h->capture) cudaStreamDestroy(h->capture);
    for (void* ptr : h->allocations) h->al.release(ptr, h->al.ctx);
    h->allocations.clear();
    delete h;
    return LBM_OK;
}

extern "C" lbm_status lbm_set_block(lbm_handle* h, int bx, int by) {
    if (!h) return LBM_ERR_ARG;
    if (bx < 1 || by < 1 || bx * by > 256 || (bx * by) % 32 != 0) return h->fail(LBM_ERR_ARG, "block shape");
    ++h->gen;
    h->bx = bx;
    h->by = by;
    return LBM_OK;
}

namespace {

// Lists the non-solid cells whose flag byte is not 0 (after the internal
// neighbour bits are set), in two parts: the cells with a rule beyond plain
// bounce-back (out, counted in count[0]) and the plain bounce-back cells,
// byte F_NEAR_SOLID alone (out_bb, count[1]).  The counters must start at 0;
// with null outputs the kernel only counts.  One atomic per warp and part; a
// warp's cells keep their order.
__global__ void k_list_special(const uint8_t* __restrict__ flags, size_t N, uint32_t* count, uint32_t* out,
                               uint32_t* out_bb) {
    const int lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    for (size_t base = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) & ~(size_t)31; base < N;
         base += (size_t)gridDim.x * blockDim.x) {
        const size_t n = base + lane;
        const uint32_t fl = n < N ? flags[n] : 0u;
        const bool bb = fl == F_NEAR_SOLID;
        const bool sp = fl != 0u && !(fl & F_WALL) && !bb;
        const uint32_t m_sp = __ballot_sync(0xffffffffu, sp), m_bb = __ballot_sync(0xffffffffu, bb);
        uint32_t at = 0, at_bb = 0;
        if (lane == 0 && m_sp) at = atomicAdd(count, (uint32_t)__popc(m_sp));
        if (lane == 0 && m_bb) at_bb = atomicAdd(count + 1, (uint32_t)__popc(m_bb));
        at = __shfl_sync(0xffffffffu, at, 0);
        at_bb = __shfl_sync(0xffffffffu, at_bb, 0);
        if (sp && out) out[at + __popc(m_sp & below)] = (uint32_t)n;
        if (bb && out_bb) out_bb[at_bb + __popc(m_bb & below)] = (uint32_t)n;
    }
}

__global__ void k_fill(float* p, size_t n, float v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

// node_u / node_rho of m listed cells (indices checked on the host, no
// duplicates); u: 3 x m component-major or NULL, rho: m or NULL
__global__ void k_scatter_nodes(const int64_t* cells, uint32_t m, const float* u, const float* rho, float* node_u,
                                float* node_rho, size_t N, int comps) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        const size_t n = (size_t)cells[k];
        if (u)
            for (int d = 0; d < 3; ++d) node_u[d * N + n] = d < comps ? u[(size_t)d * m + k] : 0.0f;
        if (rho) node_rho[n] = rho[k];
    }
}

}  // namespace

extern "C" lbm_status lbm_set_geometry(lbm_handle* h, const uint8_t* flags, const float* node_u, const float* node_rho) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    ++h->gen;
    ++h->geom_gen;
    const size_t N = h->N;
    if (!flags) {
        h->has_open_boundaries = false;
        h->release((void*&)h->special, (size_t)h->special_cap * sizeof(uint32_t));
        h->special_cap = 0;
        h->n_special = h->n_complex = 0;
        h->release((void*&)h->flags, N);
        h->release((void*&)h->walls, N * sizeof(uint32_t));
        h->release((void*&)h->node_u, 3 * N * sizeof(float));
        h->release((void*&)h->node_rho, N * sizeof(float));
        return ensure_layout(h);
    }
    bool any_moving = false, any_eq = false, any_open = false;
    for (size_t n = 0; n < N; ++n) {
        const uint32_t fl = flags[n];
        const bool wall = fl & LBM_WALL;
        if (fl & 0x80u) return h->fail(LBM_ERR_ARG, "flag bit 7 is reserved");
        if ((fl & LBM_MOVING) && !wall) return h->fail(LBM_ERR_ARG, "MOVING without WALL");
        if ((fl & LBM_FREESLIP) && (!wall || (fl & LBM_MOVING)))
            return h->fail(LBM_ERR_ARG, "FREESLIP needs WALL and excludes MOVING");
        if ((fl & 0x60u) && !(fl & LBM_FREESLIP)) return h->fail(LBM_ERR_ARG, "axis bits without FREESLIP");
        if ((fl & LBM_EQ) && (wall || (fl & LBM_OUTFLOW))) return h->fail(LBM_ERR_ARG, "EQ with WALL/OUTFLOW");
        if ((fl & LBM_OUTFLOW) && wall) return h->fail(LBM_ERR_ARG, "OUTFLOW with WALL");
        if (fl & LBM_OUTFLOW) {   // pulls as if one cell upstream in x: that cell holds populations
            const int x = (int)(n % (size_t)h->p.nx);
            if (flags[n - x + (x == 0 ? h->p.nx - 1 : x - 1)] & LBM_WALL)
                return h->fail(LBM_ERR_ARG, "OUTFLOW cell whose -x neighbour is solid");
        }
        if (h->aa() && (fl & (LBM_OUTFLOW | LBM_FREESLIP)))
            return h->fail(LBM_ERR_UNSUPPORTED, "A-A streaming supports no OUTFLOW or FREESLIP cells");
        any_moving |= (fl & LBM_MOVING) != 0;
        any_open |= (fl & (LBM_OUTFLOW | LBM_FREESLIP)) != 0;
        any_eq |= (fl & LBM_EQ) != 0;
    }
    if (!h->flags) {
        h->flags = (uint8_t*)h->alloc(N);
        if (!h->flags) return h->fail(LBM_ERR_OOM, "flags");
    }
    if (!h->walls) {
        h->walls = (uint32_t*)h->alloc(N * sizeof(uint32_t));
        if (!h->walls) return h->fail(LBM_ERR_OOM, "wall masks");
    }
    if (h->cuda(cudaMemcpyAsync(h->flags, flags, N, cudaMemcpyHostToDevice, h->stream), "flags upload"))
        return LBM_ERR_CUDA;
    h->has_open_boundaries = any_open;
    const bool need_u = node_u || any_moving || any_eq;
    const bool need_rho = node_rho || any_eq;
    if (need_u && !h->node_u) {
        h->node_u = (float*)h->alloc(3 * N * sizeof(float));
        if (!h->node_u) return h->fail(LBM_ERR_OOM, "node_u");
    }
    if (need_rho && !h->node_rho) {
        h->node_rho = (float*)h->alloc(N * sizeof(float));
        if (!h->node_rho) return h->fail(LBM_ERR_OOM, "node_rho");
    }
    if (h->node_u) {
        const int comps = h->p.velset == LBM_D2Q9 ? 2 : 3;   // D2Q9 ignores z
        if (node_u) {
            if (h->cuda(cudaMemcpyAsync(h->node_u, node_u, comps * N * sizeof(float), cudaMemcpyHostToDevice,
                                        h->stream), "node_u upload")) return LBM_ERR_CUDA;
            if (comps == 2 && h->cuda(cudaMemsetAsync(h->node_u + 2 * N, 0, N * sizeof(float), h->stream), "memset"))
                return LBM_ERR_CUDA;
        } else if (h->cuda(cudaMemsetAsync(h->node_u, 0, 3 * N * sizeof(float), h->stream), "memset")) {
            return LBM_ERR_CUDA;
        }
    }
    if (h->node_rho) {
        if (node_rho) {
            if (h->cuda(cudaMemcpyAsync(h->node_rho, node_rho, N * sizeof(float), cudaMemcpyHostToDevice, h->stream),
                        "node_rho upload")) return LBM_ERR_CUDA;
        } else {
            k_fill<<<(unsigned)std::min<size_t>((N + 255) / 256, 152 * 16), 256, 0, h->stream>>>(h->node_rho, N, 1.0f);
            if (h->cuda(cudaGetLastError(), "fill kernel")) return LBM_ERR_CUDA;
        }
    }
    {
        const int grid = (int)std::min<size_t>((N + 255) / 256, 152 * 16);
        if (h->p.velset == LBM_D2Q9)
            k_mark_neighbours<D2Q9><<<grid, 256, 0, h->stream>>>(h->flags, h->walls, h->p.nx, h->p.ny, h->p.nz);
        else if (h->p.velset == LBM_D3Q19)
            k_mark_neighbours<D3Q19><<<grid, 256, 0, h->stream>>>(h->flags, h->walls, h->p.nx, h->p.ny, h->p.nz);
        else
            k_mark_neighbours<D3Q27><<<grid, 256, 0, h->stream>>>(h->flags, h->walls, h->p.nx, h->p.ny, h->p.nz);
        if (h->cuda(cudaGetLastError(), "mark kernel")) return LBM_ERR_CUDA;
    }
    {   // list of the non-plain cells (two passes: count, then fill): the
        // cells with other rules first, then the plain bounce-back cells
        h->release((void*&)h->special, (size_t)h->special_cap * sizeof(uint32_t));
        h->special_cap = 0;
        h->n_special = h->n_complex = 0;
        uint32_t* cnt = reinterpret_cast<uint32_t*>(h->partial);   // scratch word pair
        const int grid = (int)std::min<size_t>((N + 255) / 256, 152 * 16);
        if (h->cuda(cudaMemsetAsync(cnt, 0, 2 * sizeof(uint32_t), h->stream), "memset")) return LBM_ERR_CUDA;
        k_list_special<<<grid, 256, 0, h->stream>>>(h->flags, N, cnt, nullptr, nullptr);
        if (h->cuda(cudaGetLastError(), "list kernel")) return LBM_ERR_CUDA;
        uint32_t count[2] = {0, 0};
        if (h->cuda(cudaMemcpyAsync(count, cnt, sizeof count, cudaMemcpyDeviceToHost, h->stream), "download") ||
            h->cuda(cudaStreamSynchronize(h->stream), "sync"))
            return LBM_ERR_CUDA;
        const uint32_t total = count[0] + count[1];
        if (total > 0) {
            h->special = (uint32_t*)h->alloc((size_t)total * sizeof(uint32_t));
            if (!h->special) return h->fail(LBM_ERR_OOM, "cell list");
            h->special_cap = total;
            if (h->cuda(cudaMemsetAsync(cnt, 0, 2 * sizeof(uint32_t), h->stream), "memset")) return LBM_ERR_CUDA;
            k_list_special<<<grid, 256, 0, h->stream>>>(h->flags, N, cnt, h->special, h->special + count[0]);
            if (h->cuda(cudaGetLastError(), "list kernel")) return LBM_ERR_CUDA;
        }
        h->n_special = total;
        h->n_complex = count[0];
    }
    lbm_status st2 = ensure_layout(h);
    if (st2 != LBM_OK) return st2;
    st2 = zero_solid(h);                 // solid cells hold no populations
    if (st2 != LBM_OK) return st2;
    if (h->cuda(cudaStreamSynchronize(h->stream), "sync")) return LBM_ERR_CUDA;
    return LBM_OK;
}

extern "C" lbm_status lbm_set_nodes(lbm_handle* h, int64_t count, const int64_t* cells, const float* node_u,
                                    const float* node_rho) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    ++h->gen;
    ++h->geom_gen;
    if (!h->flags) return h->fail(LBM_ERR_ARG, "lbm_set_nodes needs flags (call lbm_set_geometry first)");
    if ((st = check_cell_list(h, count, cells)) != LBM_OK) return st;
    {
        std::vector<int64_t> sorted(cells, cells + count);
        std::sort(sorted.begin(), sorted.end());
        auto dup = std::adjacent_find(sorted.begin(), sorted.end());
        if (dup != sorted.end()) return h->fail(LBM_ERR_ARG, "cell " + std::to_string(*dup) + " is listed twice");
    }
    if (count == 0 || (!node_u && !node_rho)) return LBM_OK;
    const size_t N = h->N;
    if (node_u && !h->node_u) {
        h->node_u = (float*)h->alloc(3 * N * sizeof(float));
        if (!h->node_u) return h->fail(LBM_ERR_OOM, "node_u");
        if (h->cuda(cudaMemsetAsync(h->node_u, 0, 3 * N * sizeof(float), h->stream), "memset")) return LBM_ERR_CUDA;
    }
    if (node_rho && !h->node_rho) {
        h->node_rho = (float*)h->alloc(N * sizeof(float));
        if (!h->node_rho) return h->fail(LBM_ERR_OOM, "node_rho");
        k_fill<<<(unsigned)std::min<size_t>((N + 255) / 256, 152 * 16), 256, 0, h->stream>>>(h->node_rho, N, 1.0f);
        if (h->cuda(cudaGetLastError(), "fill kernel")) return LBM_ERR_CUDA;
    }
    const int comps = h->p.velset == LBM_D2Q9 ? 2 : 3;   // D2Q9 ignores z
    const size_t m_max = std::min<size_t>(kListChunk, (size_t)count);
    TempBuffer buf(h, m_max * (sizeof(int64_t) + 4 * sizeof(float)));
    if (!buf.p) return h->fail(LBM_ERR_OOM, "node staging buffer");
    int64_t* dc = static_cast<int64_t*>(buf.p);
    float* du = reinterpret_cast<float*>(dc + m_max);
    float* dr = du + 3 * m_max;
    for (int64_t k0 = 0; k0 < count; k0 += (int64_t)m_max) {
        const size_t m = std::min<size_t>(m_max, (size_t)(count - k0));
        if (h->cuda(cudaMemcpyAsync(dc, cells + k0, m * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream), "upload"))
            return LBM_ERR_CUDA;
        if (node_u)
            for (int d = 0; d < comps; ++d)
                if (h->cuda(cudaMemcpyAsync(du + d * m, node_u + (size_t)d * count + k0, m * sizeof(float),
                                            cudaMemcpyHostToDevice, h->stream), "upload"))
                    return LBM_ERR_CUDA;
        if (node_rho && h->cuda(cudaMemcpyAsync(dr, node_rho + k0, m * sizeof(float), cudaMemcpyHostToDevice, h->stream),
                                "upload"))
            return LBM_ERR_CUDA;
        k_scatter_nodes<<<(unsigned)((m + 255) / 256), 256, 0, h->stream>>>(dc, (uint32_t)m, node_u ? du : nullptr,
                                                                           node_rho ? dr : nullptr, h->node_u,
                                                                           h->node_rho, N, comps);
        if (h->cuda(cudaGetLastError(), "scatter kernel")) return LBM_ERR_CUDA;
        if (h->cuda(cudaStreamSynchronize(h->stream), "sync")) return LBM_ERR_CUDA;   // staging is reused
    }
    return LBM_OK;
}

namespace {

// zero every population copy and run the put kernel over z-chunks;
// `upload(z0, z1, dev)` stages the chunk's input doubles into dev
template <class R, class Up>
lbm_status put_all(lbm_handle* h, const Relax<R>& k, int setf, int per_cell, Up upload) {
    const size_t fbytes = h->fbytes();
    ++h->gen;
    for (int c = 0; c < (h->aa() ? 1 : 2); ++c)
        if (h->cuda(cudaMemsetAsync(h->f[c], 0, fbytes, h->stream), "memset")) return LBM_ERR_CUDA;
    h->chunked = want_chunked(h) ? 1 : 0;   // the populations are rewritten: take the best layout
    const int chunk = h->planes_per_chunk(per_cell);
    for (int z0 = 0; z0 < h->p.nz; z0 += chunk) {
        const int z1 = std::min(h->p.nz, z0 + chunk);
        PutArgs<R> pa{};
        pa.a = h->args(k, 1);   // dst = f[0] for both schemes
        pa.a.dst = h->f[0];
        pa.z0 = z0;
        pa.z1 = z1;
        upload(z0, z1, pa.in);
        if (h->sticky) return LBM_ERR_CUDA;
        const size_t count = (size_t)h->plane() * (z1 - z0);
        Launch L;
        L.block = dim3(256);
        L.grid = dim3((unsigned)std::min<size_t>((count + 255) / 256, 152 * 32));
        L.stream = h->stream;
        if (h->cuda(h->ks->put[(h->aa() ? 1 : 0) | (h->chunked ? 2 : 0)](&pa, setf, L), "put kernel"))
            return LBM_ERR_CUDA;
        // the next chunk's upload into the staging buffer follows this kernel in stream order
    }
    if (h->cuda(cudaStreamSynchronize(h->stream), "sync")) return LBM_ERR_CUDA;
    h->t = 0;
    h->cur = 0;
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_set_rho_u(lbm_handle* h, const double* rho, const double* ux, const double* uy, const double* uz) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    Staging staging(h);
    if (!staging.ok()) return h->fail(LBM_ERR_OOM, "staging buffer");
    const double* src[4] = {rho, ux, uy, uz};
    auto upload = [&](int z0, int z1, const double** in) {
        const size_t count = (size_t)h->plane() * (z1 - z0);
        const size_t off = (size_t)h->plane() * z0;
        for (int c = 0; c < 4; ++c) {
            in[c] = nullptr;
            if (!src[c]) continue;
            double* d = h->scratch + c * count;
            if (h->cuda(cudaMemcpyAsync(d, src[c] + off, count * sizeof(double), cudaMemcpyHostToDevice, h->stream),
                        "fields upload")) return;
            in[c] = d;
        }
    };
    return h->fp64() ? put_all(h, h->kd, 0, 4, upload) : put_all(h, h->kf, 0, 4, upload);
}

extern "C" lbm_status lbm_set_f(lbm_handle* h, const double* f) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    Staging staging(h);
    if (!staging.ok()) return h->fail(LBM_ERR_OOM, "staging buffer");
    if (!f) return h->fail(LBM_ERR_ARG, "f is NULL");
    auto upload = [&](int z0, int z1, const double** in) {
        const size_t count = (size_t)h->plane() * (z1 - z0);
        const size_t off = (size_t)h->plane() * z0;
        for (int i = 0; i < h->q; ++i)
            if (h->cuda(cudaMemcpyAsync(h->scratch + i * count, f + (size_t)i * h->N + off, count * sizeof(double),
                                        cudaMemcpyHostToDevice, h->stream), "f upload")) return;
        in[0] = h->scratch;
        in[1] = in[2] = in[3] = nullptr;
    };
    return h->fp64() ? put_all(h, h->kd, 1, h->q, upload) : put_all(h, h->kf, 1, h->q, upload);
}

namespace {

// index of the staged kernel that applies to h, or -1
int staged_index(const lbm_handle* h) {
    if (h->flags || h->aa() || h->fp64() || h->p.velset != LBM_D3Q19 || !h->idx32()) return -1;
    const int idx = h->p.nx == 128 ? 0 : (h->p.nx == 256 ? 1 : (h->p.nx == 512 ? 2 : -1));
    if (idx < 0 || !h->ks->staged[idx]) return -1;
    return idx;
}

// the chunked layout: 16-bit storage, FP32 arithmetic, nx a multiple of 64
// (A-B or A-A, with or without flags, any size)
bool chunk_eligible(const lbm_handle* h) {
    return !h->fp64() && h->sb == 2 && (h->p.nx % lbm::CHUNK) == 0 && h->ks->pair_chunked[0][0];
}
bool want_chunked(const lbm_handle* h) {
    if (h->force_chunked && !h->fp64() && h->sb == 2 && h->ks->step_ch[0]) return true;
    return chunk_eligible(h) && (h->variant == LBM_VARIANT_AUTO || h->variant == LBM_VARIANT_PAIRED);
}

bool pair_applies(const lbm_handle* h) {
    return !h->flags && !h->aa() && !h->fp64() && h->sb == 2 && (h->p.nx % 2) == 0 && h->idx32() &&
           (h->bx % 32) == 0 && h->ks->pair;
}

// kernel variant lbm_step launches for h
int variant_in_use(const lbm_handle* h) {
    if (h->chunked) return LBM_VARIANT_PAIRED;
    if (h->variant == LBM_VARIANT_STAGED && staged_index(h) >= 0) return LBM_VARIANT_STAGED;
    // without the chunked layout the paired kernel pays off only with hardware
    // conversions (FP16, FP16S); AUTO keeps the software codecs on GENERIC
    const bool hw = h->p.storage == LBM_FP16 || h->p.storage == LBM_FP16S;
    if ((h->variant == LBM_VARIANT_PAIRED || (h->variant == LBM_VARIANT_AUTO && hw)) && pair_applies(h))
        return LBM_VARIANT_PAIRED;
    return LBM_VARIANT_GENERIC;
}

// copies the population codes between the SoA and the chunked layout
template <class V>
__global__ void k_relayout(const uint16_t* __restrict__ src, uint16_t* __restrict__ dst, uint32_t N,
                           int to_chunked) {
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < V::Q; ++i) {
            const size_t soa = (size_t)i * N + n, ch = lbm::chunk_elem<V>(i, n);
            if (to_chunked) dst[ch] = src[soa];
            else dst[soa] = src[ch];
        }
    }
}

// zeroes the populations of solid cells (SoA, or chunked: element
// ((n/64) q + i) 64 + n%64)
template <class T>
__global__ void k_zero_solid(const uint8_t* __restrict__ flags, T* f, int q, uint32_t N, int chunked) {
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x)
        if (flags[n] & lbm::F_WALL)
            for (int i = 0; i < q; ++i) {
                const size_t e = chunked ? ((size_t)(n >> 6) * q + i) * lbm::CHUNK + (n & (lbm::CHUNK - 1))
                                         : (size_t)i * N + n;
                f[e] = T(0);
            }
}

lbm_status zero_solid(lbm_handle* h) {
    const unsigned grid = (unsigned)std::min<size_t>((h->N + 255) / 256, 152 * 32);
    for (int c = 0; c < (h->aa() ? 1 : 2); ++c) {
        const int ch = h->chunked;
        if (h->sb == 8) k_zero_solid<double><<<grid, 256, 0, h->stream>>>(h->flags, (double*)h->f[c], h->q, (uint32_t)h->N, ch);
        else if (h->sb == 4) k_zero_solid<float><<<grid, 256, 0, h->stream>>>(h->flags, (float*)h->f[c], h->q, (uint32_t)h->N, ch);
        else k_zero_solid<uint16_t><<<grid, 256, 0, h->stream>>>(h->flags, (uint16_t*)h->f[c], h->q, (uint32_t)h->N, ch);
        if (h->cuda(cudaGetLastError(), "zero kernel")) return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

// brings the stored populations into the layout the current settings call for
lbm_status ensure_layout(lbm_handle* h) {
    const int want = want_chunked(h) ? 1 : 0;
    if (want == h->chunked) return LBM_OK;
    ++h->gen;
    // A-B: into the other copy; A-A (one copy): through a transient copy of it
    const size_t fbytes = h->fbytes();
    TempBuffer tmp(h, h->aa() ? fbytes : 0);
    if (h->aa()) {
        if (!tmp.p) return h->fail(LBM_ERR_OOM, "relayout buffer");
        if (h->cuda(cudaMemcpyAsync(tmp.p, h->f[0], fbytes, cudaMemcpyDeviceToDevice, h->stream), "copy"))
            return LBM_ERR_CUDA;
    }
    const uint16_t* src = h->aa() ? (const uint16_t*)tmp.p : (const uint16_t*)h->f[h->cur];
    uint16_t* dst = h->aa() ? (uint16_t*)h->f[0] : (uint16_t*)h->f[1 - h->cur];
    const unsigned grid = (unsigned)std::min<size_t>((h->N + 255) / 256, 152 * 32);
    if (h->p.velset == LBM_D2Q9) k_relayout<D2Q9><<<grid, 256, 0, h->stream>>>(src, dst, (uint32_t)h->N, want);
    else if (h->p.velset == LBM_D3Q19) k_relayout<D3Q19><<<grid, 256, 0, h->stream>>>(src, dst, (uint32_t)h->N, want);
    else k_relayout<D3Q27><<<grid, 256, 0, h->stream>>>(src, dst, (uint32_t)h->N, want);
    if (h->cuda(cudaGetLastError(), "relayout kernel")) return LBM_ERR_CUDA;
    if (!h->aa()) h->cur = 1 - h->cur;
    h->chunked = want;
    return LBM_OK;
}

template <class R> lbm_status launch_one_step(lbm_handle* h, const Relax<R>& k, cudaStream_t s) {
    const int scheme = h->scheme_now();
    StepArgs<R> a = h->args(k, h->aa() ? 0 : h->cur);
    const int variant = variant_in_use(h);
    lbm_status st;
    if (h->chunked && (h->p.nx % lbm::CHUNK) != 0) {
        // chunked layout forced by an ensemble on rows that are not whole
        // chunks: the generic kernel with chunked addressing, then the list
        st = h->cuda(h->ks->step_ch[scheme](&a, h->step_launch(s)), "step kernel");
        if (st == LBM_OK && h->flags && h->n_complex > 0) {
            Launch B;
            B.block = dim3(256);
            B.grid = dim3((h->n_complex + 255) / 256);
            B.stream = s;
            st = h->cuda(h->ks->list_chunked[scheme](&a, h->special, h->n_complex, B), "list kernel");
        }
    } else if (h->chunked) {
        Launch L;
        L.block = dim3(32, 8, 1);
        L.grid = dim3(h->p.nx / lbm::CHUNK, (h->p.ny + 7) / 8, h->p.nz);
        L.stream = s;
        // prefetch distance: about one and a half waves of blocks (3 resident
        // per SM, 2 for D3Q27), as rows of 8 (one block row) split into planes
        // and rows
        const long ahead = (h->q > 19 ? 2L : 3L) * h->num_sms * 3 / 2;
        const long rows = (ahead + L.grid.x - 1) / L.grid.x * 8;
        a.pf = (int)(rows / h->p.ny);
        a.pf_y = (int)(rows % h->p.ny);
        st = h->cuda(h->ks->pair_chunked[scheme][h->flags ? 1 : 0](&a, L), "chunked step kernel");
        // the non-plain cells; the paired kernel updates the plain bounce-back
        // cells itself except in the odd A-A half
        const uint32_t nl = scheme == lbm::SCHEME_AA_PP ? h->n_special : h->n_complex;
        if (st == LBM_OK && h->flags && nl > 0) {
            Launch B;
            B.block = dim3(256);
            B.grid = dim3((nl + 255) / 256);
            B.stream = s;
            st = h->cuda(h->ks->list_chunked[scheme](&a, h->special, nl, B), "list kernel");
        }
    } else if (variant == LBM_VARIANT_PAIRED) {
        Launch L;
        L.block = dim3(h->bx, h->by, 1);
        L.grid = dim3((h->p.nx / 2 + h->bx - 1) / h->bx, (h->p.ny + h->by - 1) / h->by, h->p.nz);
        L.stream = s;
        st = h->cuda(h->ks->pair(&a, L), "paired step kernel");
    } else if (variant == LBM_VARIANT_STAGED) {
        const int si = staged_index(h);
        const int rows = h->ks->staged_rows[si];
        const int tiles_y = (h->p.ny + rows - 1) / rows;
        const int grid = std::min(tiles_y * h->p.nz, 2 * h->num_sms);
        st = h->cuda(h->ks->staged[si](&a, grid, tiles_y, h->status, s), "staged step kernel");
    } else {
        st = h->cuda(h->ks->step[scheme][h->flags ? 1 : 0][h->idx32() ? 1 : 0](&a, h->step_launch(s)),
                     "step kernel");
        // the non-plain cells except the plain bounce-back ones, which the
        // step kernel updates itself
        if (st == LBM_OK && h->flags && h->n_complex > 0) {
            Launch L;
            L.block = dim3(256);
            L.grid = dim3((h->n_complex + 255) / 256);
            L.stream = s;
            st = h->cuda(h->ks->list[scheme][h->idx32() ? 1 : 0](&a, h->special, h->n_complex, L), "list kernel");
        }
    }
    if (st != LBM_OK) return st;
    if (!h->aa()) h->cur ^= 1;
    h->t += 1;
    return LBM_OK;
}

}  // namespace

lbm_status lbm_internal_check_status(lbm_handle* h) { return check_status(h); }
lbm_status lbm_internal_ensure_layout(lbm_handle* h) { return ensure_layout(h); }

lbm_status lbm_internal_step(lbm_handle* h, cudaStream_t s) {
    return h->fp64() ? launch_one_step(h, h->kd, s) : launch_one_step(h, h->kf, s);
}

namespace {

// Lattices up to kGraphCells cells, whose steps are short enough for launch
// overhead to show, replay runs of kStepGraph steps from a CUDA graph.
constexpr int kStepGraph = 32;                       // even: cur and t & 1 return to their start values
constexpr size_t kGraphCells = size_t(1) << 23;

// the graph of kStepGraph steps from the current state, captured if missing
// or stale; *out stays NULL where the runtime declines the capture
lbm_status step_graph(lbm_handle* h, cudaGraphExec_t* out) {
    *out = nullptr;
    const int c = h->cur, par = (int)(h->t & 1);
    if (h->graph[c][par] && h->graph_gen[c][par] == h->gen) {
        *out = h->graph[c][par];
        return LBM_OK;
    }
    if (h->graph[c][par]) {
        if (h->cuda(cudaGraphExecDestroy(h->graph[c][par]), "graph destroy")) return LBM_ERR_CUDA;
        h->graph[c][par] = nullptr;
    }
    if (!h->capture && h->cuda(cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking), "capture stream"))
        return LBM_ERR_CUDA;
    // capture on the private stream (nothing runs); the replays go to h->stream.
    // A capture the runtime refuses leaves the steps to plain launches.
    if (cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return LBM_OK;
    }
    const int64_t t0 = h->t;
    const int c0 = h->cur;
    lbm_status st = LBM_OK;
    for (int k = 0; k < kStepGraph && st == LBM_OK; ++k) st = lbm_internal_step(h, h->capture);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->capture, &graph);
    h->t = t0;
    h->cur = c0;
    if (st != LBM_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (st != LBM_OK) return st;   // a launch failed: reported like an uncaptured one
        cudaGetLastError();
        return LBM_OK;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e2 = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess) {
        cudaGetLastError();
        return LBM_OK;
    }
    h->graph[c][par] = exec;
    h->graph_gen[c][par] = h->gen;
    *out = exec;
    return LBM_OK;
}

}  // namespace

namespace {

lbm_status reduce_any(lbm_handle* h, double* mass, double* energy);

// nsteps steps without divergence checks
lbm_status step_run(lbm_handle* h, int64_t nsteps) {
    lbm_status st = LBM_OK;
    int64_t s = 0;
    if (h->N <= kGraphCells && nsteps >= 2 * kStepGraph) {
        cudaGraphExec_t g = nullptr;
        if ((st = step_graph(h, &g)) != LBM_OK) return st;
        for (; g && s + kStepGraph <= nsteps; s += kStepGraph) {
            if (h->cuda(cudaGraphLaunch(g, h->stream), "graph launch")) return LBM_ERR_CUDA;
            h->t += kStepGraph;   // h->cur is back at its start value
        }
    }
    for (; s < nsteps; ++s) {
        st = lbm_internal_step(h, h->stream);
        if (st != LBM_OK) return st;
    }
    return LBM_OK;
}

// the FP64 check of lbm_set_divergence_check at the current step
lbm_status divergence_check(lbm_handle* h) {
    double mass = 0.0, energy = 0.0;
    const lbm_status st = reduce_any(h, &mass, &energy);
    if (st == LBM_ERR_DIVERGED || (st == LBM_OK && h->check_tol > 0.0 &&
                                   std::fabs(mass - h->check_mass0) > h->check_tol * std::fabs(h->check_mass0))) {
        h->err = "diverged at step " + std::to_string(h->t) + ": mass " + std::to_string(mass) + " (set " +
                 std::to_string(h->check_mass0) + "), kinetic energy " + std::to_string(energy);
        return LBM_ERR_DIVERGED;
    }
    return st;
}

}  // namespace

extern "C" lbm_status lbm_step(lbm_handle* h, int64_t nsteps) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    if (nsteps < 0) return h->fail(LBM_ERR_ARG, "negative step count");
    if (h->check_every <= 0) return step_run(h, nsteps);
    // runs up to the next multiple of check_every of the step counter, each followed by the check
    while (nsteps > 0) {
        const int64_t to_check = h->check_every - (h->t % h->check_every);
        const int64_t n = std::min(nsteps, to_check);
        if ((st = step_run(h, n)) != LBM_OK) return st;
        nsteps -= n;
        if (h->t % h->check_every == 0 && (st = divergence_check(h)) != LBM_OK) return st;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_set_divergence_check(lbm_handle* h, int64_t every, double mass_tol) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    if (every < 0 || !std::isfinite(mass_tol)) return h->fail(LBM_ERR_ARG, "divergence check: every < 0 or mass_tol");
    h->check_every = every;
    h->check_tol = mass_tol;
    if (every == 0) return LBM_OK;
    double mass = 0.0, energy = 0.0;
    st = reduce_any(h, &mass, &energy);
    h->check_mass0 = mass;
    if (st != LBM_OK) h->check_every = 0;
    return st;
}

namespace {

template <class R>
lbm_status probe_chunks(lbm_handle* h, const Relax<R>& k, int mode, int per_cell,
                        const std::function<lbm_status(int, int, size_t)>& download) {
    const int chunk = h->planes_per_chunk(per_cell);
    for (int z0 = 0; z0 < h->p.nz; z0 += chunk) {
        const int z1 = std::min(h->p.nz, z0 + chunk);
        ProbeArgs<R> pa{};
        pa.a = h->args(k, h->aa() ? 0 : h->cur);
        pa.z0 = z0;
        pa.z1 = z1;
        pa.out = h->scratch;
        pa.partial = h->partial;
        const size_t count = (size_t)h->plane() * (z1 - z0);
        Launch L;
        L.block = dim3(256);
        L.grid = dim3((unsigned)std::min<size_t>((count + 255) / 256, 152 * 32));
        L.stream = h->stream;
        if (h->cuda(h->ks->probe[h->layout_now()](&pa, mode, L), "probe kernel")) return LBM_ERR_CUDA;
        lbm_status st = download(z0, z1, count);
        if (st != LBM_OK) return st;
    }
    return h->cuda(cudaStreamSynchronize(h->stream), "sync");
}

}  // namespace

extern "C" lbm_status lbm_get_rho_u(lbm_handle* h, double* rho, double* ux, double* uy, double* uz) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    Staging staging(h);
    if (!staging.ok()) return h->fail(LBM_ERR_OOM, "staging buffer");
    double* dst[4] = {rho, ux, uy, uz};
    auto download = [&](int z0, int, size_t count) -> lbm_status {
        const size_t off = (size_t)h->plane() * z0;
        for (int c = 0; c < 4; ++c)
            if (dst[c] && h->cuda(cudaMemcpyAsync(dst[c] + off, h->scratch + c * count, count * sizeof(double),
                                                  cudaMemcpyDeviceToHost, h->stream), "fields download"))
                return LBM_ERR_CUDA;
        return LBM_OK;   // the next chunk's probe follows these copies in stream order
    };
    st = h->fp64() ? probe_chunks(h, h->kd, PROBE_FIELDS, 4, download)
                   : probe_chunks(h, h->kf, PROBE_FIELDS, 4, download);
    return st == LBM_OK ? check_status(h) : st;
}

extern "C" lbm_status lbm_get_f(lbm_handle* h, double* f) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    Staging staging(h);
    if (!staging.ok()) return h->fail(LBM_ERR_OOM, "staging buffer");
    if (!f) return h->fail(LBM_ERR_ARG, "f is NULL");
    auto download = [&](int z0, int, size_t count) -> lbm_status {
        const size_t off = (size_t)h->plane() * z0;
        for (int i = 0; i < h->q; ++i)
            if (h->cuda(cudaMemcpyAsync(f + (size_t)i * h->N + off, h->scratch + i * count, count * sizeof(double),
                                        cudaMemcpyDeviceToHost, h->stream), "f download"))
                return LBM_ERR_CUDA;
        return LBM_OK;   // the next chunk's probe follows these copies in stream order
    };
    st = h->fp64() ? probe_chunks(h, h->kd, PROBE_F, h->q, download)
                   : probe_chunks(h, h->kf, PROBE_F, h->q, download);
    return st == LBM_OK ? check_status(h) : st;
}

namespace {

// Probe kernel over a list of cells, in chunks of at most kListChunk cells;
// download(k0, m, out) copies m cells' results (per_cell x m doubles) out.
template <class R>
lbm_status probe_list(lbm_handle* h, const Relax<R>& k, int mode, int per_cell, int64_t count, const int64_t* cells,
                      const std::function<lbm_status(int64_t, size_t, const double*)>& download) {
    const size_t m_max = std::min<size_t>(kListChunk, (size_t)count);
    TempBuffer buf(h, m_max * (per_cell + 1) * sizeof(double));
    if (!buf.p) return h->fail(LBM_ERR_OOM, "probe buffer");
    double* out = static_cast<double*>(buf.p);
    int64_t* dev_cells = reinterpret_cast<int64_t*>(out + (size_t)per_cell * m_max);
    for (int64_t k0 = 0; k0 < count; k0 += (int64_t)m_max) {
        const size_t m = std::min<size_t>(m_max, (size_t)(count - k0));
        if (h->cuda(cudaMemcpyAsync(dev_cells, cells + k0, m * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream),
                    "cell list upload")) return LBM_ERR_CUDA;
        ProbeArgs<R> pa{};
        pa.a = h->args(k, h->aa() ? 0 : h->cur);
        pa.out = out;
        pa.partial = h->partial;
        pa.cells = dev_cells;
        pa.ncells = (uint32_t)m;
        Launch L;
        L.block = dim3(256);
        L.grid = dim3((unsigned)((m + 255) / 256));
        L.stream = h->stream;
        if (h->cuda(h->ks->probe[h->layout_now()](&pa, mode, L), "probe kernel")) return LBM_ERR_CUDA;
        lbm_status st = download(k0, m, out);
        if (st != LBM_OK) return st;
    }
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_get_f_cells(lbm_handle* h, int64_t count, const int64_t* cells, double* f) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    if (count > 0 && !f) return h->fail(LBM_ERR_ARG, "f is NULL");
    if ((st = check_cell_list(h, count, cells)) != LBM_OK) return st;
    if (count == 0) return LBM_OK;
    auto download = [&](int64_t k0, size_t m, const double* out) -> lbm_status {
        for (int i = 0; i < h->q; ++i)
            if (h->cuda(cudaMemcpyAsync(f + (size_t)i * count + k0, out + (size_t)i * m, m * sizeof(double),
                                        cudaMemcpyDeviceToHost, h->stream), "f download"))
                return LBM_ERR_CUDA;
        return h->cuda(cudaStreamSynchronize(h->stream), "sync");
    };
    st = h->fp64() ? probe_list(h, h->kd, PROBE_F, h->q, count, cells, download)
                   : probe_list(h, h->kf, PROBE_F, h->q, count, cells, download);
    return st == LBM_OK ? check_status(h) : st;
}

extern "C" lbm_status lbm_get_rho_u_cells(lbm_handle* h, int64_t count, const int64_t* cells, double* rho,
                                          double* ux, double* uy, double* uz) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    if ((st = check_cell_list(h, count, cells)) != LBM_OK) return st;
    if (count == 0) return LBM_OK;
    double* dst[4] = {rho, ux, uy, uz};
    auto download = [&](int64_t k0, size_t m, const double* out) -> lbm_status {
        for (int c = 0; c < 4; ++c)
            if (dst[c] && h->cuda(cudaMemcpyAsync(dst[c] + k0, out + (size_t)c * m, m * sizeof(double),
                                                  cudaMemcpyDeviceToHost, h->stream), "fields download"))
                return LBM_ERR_CUDA;
        return h->cuda(cudaStreamSynchronize(h->stream), "sync");
    };
    st = h->fp64() ? probe_list(h, h->kd, PROBE_FIELDS, 4, count, cells, download)
                   : probe_list(h, h->kf, PROBE_FIELDS, 4, count, cells, download);
    return st == LBM_OK ? check_status(h) : st;
}

namespace {

// sums the per-block partials in a fixed order (one warp)
__global__ void k_sum_partials(const double* partial, int blocks, double* out) {
    double m = 0.0, e = 0.0;
    for (int b = threadIdx.x; b < blocks; b += 32) {
        m += partial[2 * b];
        e += partial[2 * b + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m += __shfl_down_sync(0xffffffffu, m, o);
        e += __shfl_down_sync(0xffffffffu, e, o);
    }
    if (threadIdx.x == 0) { out[0] = m; out[1] = e; }
}

template <class R> lbm_status reduce_impl(lbm_handle* h, const Relax<R>& k, double* mass, double* energy) {
    ProbeArgs<R> pa{};
    pa.a = h->args(k, h->aa() ? 0 : h->cur);
    pa.z0 = 0;
    pa.z1 = h->p.nz;
    pa.out = nullptr;
    pa.partial = h->partial;
    Launch L;
    L.block = dim3(256);
    L.grid = dim3((unsigned)std::min<size_t>((h->N + 255) / 256, kReduceBlocks));
    L.stream = h->stream;
    if (h->cuda(h->ks->probe[h->layout_now()](&pa, PROBE_REDUCE, L), "reduce kernel")) return LBM_ERR_CUDA;
    double* out = h->partial + 2 * kReduceBlocks;
    k_sum_partials<<<1, 32, 0, h->stream>>>(h->partial, (int)L.grid.x, out);
    if (h->cuda(cudaGetLastError(), "sum kernel")) return LBM_ERR_CUDA;
    double res[2];
    if (h->cuda(cudaMemcpyAsync(res, out, sizeof res, cudaMemcpyDeviceToHost, h->stream), "download")) return LBM_ERR_CUDA;
    if (h->cuda(cudaStreamSynchronize(h->stream), "sync")) return LBM_ERR_CUDA;
    if (check_status(h) != LBM_OK) return LBM_ERR_TIMEOUT;
    if (mass) *mass = res[0];
    if (energy) *energy = res[1];
    if (!std::isfinite(res[0]) || !std::isfinite(res[1])) return h->fail(LBM_ERR_DIVERGED, "non-finite mass or energy");
    return LBM_OK;
}

}  // namespace

namespace {
lbm_status reduce_any(lbm_handle* h, double* mass, double* energy) {
    return h->fp64() ? reduce_impl(h, h->kd, mass, energy) : reduce_impl(h, h->kf, mass, energy);
}
}  // namespace

extern "C" lbm_status lbm_reduce(lbm_handle* h, double* mass, double* kinetic_energy) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    return reduce_any(h, mass, kinetic_energy);
}

namespace {

// One thread waits on an mbarrier that nothing ever arrives on, with the same
// bounded wait as the bulk-copy kernels; when it runs out, the thread reports
// it through the handle's status word.
__global__ void k_wait_unarrived(int* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        lbm::mbar_init(&bar, 1);
        lbm::mbar_fence_init();
        if (!lbm::mbar_wait(&bar, 0)) atomicExch(status, 1);
    }
}

}  // namespace

extern "C" lbm_status lbm_selftest_wait_timeout(lbm_handle* h) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    k_wait_unarrived<<<1, 32, 0, h->stream>>>(h->status);
    if (h->cuda(cudaGetLastError(), "wait kernel")) return LBM_ERR_CUDA;
    if (h->cuda(cudaStreamSynchronize(h->stream), "sync")) return LBM_ERR_CUDA;
    return check_status(h);
}

extern "C" lbm_status lbm_get_info(const lbm_handle* h, lbm_info* info) {
    if (!h || !info) return LBM_ERR_ARG;
    info->q = h->q;
    info->cells = (int64_t)h->N;
    info->step = h->t;
    info->bytes_per_population = h->sb;
    info->has_flags = h->flags ? 1 : 0;
    info->device_bytes = h->device_bytes;
    info->ddf[0] = h->aa() ? h->f[0] : h->f[h->cur];
    info->ddf[1] = h->aa() ? nullptr : h->f[1 - h->cur];
    info->layout = h->chunked ? LBM_LAYOUT_CHUNKED : LBM_LAYOUT_SOA;
    info->scheme = h->p.scheme;
    return LBM_OK;
}


extern "C" lbm_status lbm_autotune(lbm_handle* h, int trial_steps, int* bx_out, int* by_out) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    if (trial_steps < 1) return h->fail(LBM_ERR_ARG, "trial_steps < 1");
    cudaEvent_t ev[2];
    if (h->cuda(cudaEventCreate(&ev[0]), "event") || h->cuda(cudaEventCreate(&ev[1]), "event")) return LBM_ERR_CUDA;
    // 2 untimed steps, then trial_steps timed on the lattice's stream
    auto trial = [&](float* ms) -> lbm_status {
        lbm_status s2 = lbm_step(h, 2);
        if (s2 != LBM_OK) return s2;
        cudaEventRecord(ev[0], h->stream);
        if ((s2 = lbm_step(h, trial_steps)) != LBM_OK) return s2;
        cudaEventRecord(ev[1], h->stream);
        if (h->cuda(cudaEventSynchronize(ev[1]), "event sync")) return LBM_ERR_CUDA;
        return h->cuda(cudaEventElapsedTime(ms, ev[0], ev[1]), "event time");
    };
    // 0. lattices created with LBM_STREAM_AUTO: A-B against in-place A-A
    //    (with the default variant), where the switch is allowed
    if (h->scheme_auto && !(h->t & 1) && !h->has_open_boundaries) {
        const int s0 = h->p.scheme, s1 = s0 == LBM_STREAM_AB ? LBM_STREAM_AA : LBM_STREAM_AB;
        float m0 = 0.f, m1 = 1e30f;
        if ((st = trial(&m0)) != LBM_OK) { cudaEventDestroy(ev[0]); cudaEventDestroy(ev[1]); return st; }
        if (trial_steps & 1) lbm_step(h, 1);   // back to an even step count
        if (lbm_set_scheme(h, s1) == LBM_OK) {
            if ((st = trial(&m1)) != LBM_OK) { cudaEventDestroy(ev[0]); cudaEventDestroy(ev[1]); return st; }
            if (trial_steps & 1) lbm_step(h, 1);
            if (m0 <= m1 && (st = lbm_set_scheme(h, s0)) != LBM_OK) {
                cudaEventDestroy(ev[0]);
                cudaEventDestroy(ev[1]);
                return st;
            }
        } else {
            h->err.clear();   // no memory for the second copy: stay
        }
    }
    // 1. the kernel variant, and with it the layout: GENERIC on the structure
    //    of arrays, PAIRED (chunked layout where nx is a multiple of 64),
    //    STAGED; those that do not apply to this lattice are skipped
    float best = 1e30f;
    int best_v = LBM_VARIANT_GENERIC;
    for (int v : {LBM_VARIANT_GENERIC, LBM_VARIANT_PAIRED, LBM_VARIANT_STAGED}) {
        if ((st = lbm_set_variant(h, v)) != LBM_OK) break;
        if (variant_in_use(h) != v) continue;
        float ms = 0.f;
        if ((st = trial(&ms)) != LBM_OK) break;
        if (ms < best) { best = ms; best_v = v; }
    }
    if (st == LBM_OK) st = lbm_set_variant(h, best_v);
    // 2. the thread-block shape, for the kernels that take one (the generic
    //    kernel and the paired kernel on the structure of arrays)
    static const int shapes[][2] = {{128, 2}, {256, 1}, {64, 4}, {32, 8}, {64, 2}, {128, 1}, {32, 4}};
    int bb[2] = {h->bx, h->by};
    const int vu = st == LBM_OK ? variant_in_use(h) : -1;
    if (vu == LBM_VARIANT_GENERIC || (vu == LBM_VARIANT_PAIRED && !h->chunked)) {
        best = 1e30f;
        for (const auto& sh : shapes) {
            h->bx = sh[0];
            h->by = sh[1];
            ++h->gen;   // the launches change: no graph of another shape is replayed
            if (variant_in_use(h) != vu) continue;   // a width the paired kernel does not take
            float ms = 0.f;
            if ((st = trial(&ms)) != LBM_OK) break;
            if (ms < best) { best = ms; bb[0] = sh[0]; bb[1] = sh[1]; }
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    h->bx = bb[0];
    h->by = bb[1];
    ++h->gen;
    if (bx_out) *bx_out = bb[0];
    if (by_out) *by_out = bb[1];
    return st;
}

namespace {

// swaps slots p and p+1 (odd p: opposite directions) of every cell, in the
// SoA or the chunked layout; the rest slot stays
template <class T>
__global__ void k_swap_slots(T* f, int q, uint32_t N, int chunked) {
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x)
        for (int p = 1; p < q; p += 2) {
            const size_t a = chunked ? ((size_t)(n >> 6) * q + p) * lbm::CHUNK + (n & (lbm::CHUNK - 1))
                                     : (size_t)p * N + n;
            const size_t b = chunked ? a + lbm::CHUNK : a + N;
            const T t = f[a];
            f[a] = f[b];
            f[b] = t;
        }
}

}  // namespace

extern "C" lbm_status lbm_set_scheme(lbm_handle* h, int scheme) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    if (scheme != LBM_STREAM_AB && scheme != LBM_STREAM_AA) return h->fail(LBM_ERR_ARG, "scheme");
    if (scheme == h->p.scheme) return LBM_OK;
    if (h->t & 1) return h->fail(LBM_ERR_STATE, "the streaming scheme can change after an even number of steps only");
    if (scheme == LBM_STREAM_AA && h->has_open_boundaries)
        return h->fail(LBM_ERR_UNSUPPORTED, "A-A streaming supports no OUTFLOW or FREESLIP cells");
    const size_t fbytes = h->fbytes();
    if (scheme == LBM_STREAM_AB) {   // a second copy first: failing leaves the lattice as it was
        void* other = h->alloc(fbytes);
        if (!other) return h->fail(LBM_ERR_OOM, "second population copy");
        h->f[1] = other;
    }
    void* live = scheme == LBM_STREAM_AA ? h->f[h->cur] : h->f[0];
    // A-B after an even step count: slot i of cell x holds what x streams out
    // along i; A-A before its odd half holds the same value in slot opposite(i)
    const unsigned grid = (unsigned)std::min<size_t>((h->N + 255) / 256, 152 * 32);
    const int ch = h->chunked;
    if (h->sb == 8) k_swap_slots<double><<<grid, 256, 0, h->stream>>>((double*)live, h->q, (uint32_t)h->N, ch);
    else if (h->sb == 4) k_swap_slots<float><<<grid, 256, 0, h->stream>>>((float*)live, h->q, (uint32_t)h->N, ch);
    else k_swap_slots<uint16_t><<<grid, 256, 0, h->stream>>>((uint16_t*)live, h->q, (uint32_t)h->N, ch);
    if (h->cuda(cudaGetLastError(), "swap kernel")) return LBM_ERR_CUDA;
    if (scheme == LBM_STREAM_AA) {
        void* spare = h->f[1 - h->cur];
        h->f[0] = live;
        h->f[1] = nullptr;
        h->release(spare, fbytes);   // stream-ordered: the swap kernel does not touch it
    } else {
        // the copy the next step writes must hold zero populations for solid cells
        if (h->cuda(cudaMemsetAsync(h->f[1], 0, fbytes, h->stream), "memset")) return LBM_ERR_CUDA;
    }
    h->cur = 0;
    h->p.scheme = scheme;
    ++h->gen;
    return ensure_layout(h);
}

extern "C" lbm_status lbm_set_variant(lbm_handle* h, int variant) {
    if (!h) return LBM_ERR_ARG;
    if (variant < LBM_VARIANT_AUTO || variant > LBM_VARIANT_PAIRED) return h->fail(LBM_ERR_ARG, "variant");
    ++h->gen;
    h->variant = variant;
    return ensure_layout(h);
}

extern "C" int lbm_get_variant(const lbm_handle* h) { return h ? variant_in_use(h) : -1; }
