// Host implementation of the C ABI declared in include/lbm.h.
// Validates arguments, owns device memory through the caller's allocator,
// moves data in bounded chunks and launches the kernels of lbm_kernels.cuh.
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
    static KernelSet table[3][2][10][2];
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
    k.cs = (R)(1.0 / std::sqrt(3.0));
    for (int a = 0; a < 3; ++a) k.F[a] = (R)p.force[a];
    k.force = (p.force[0] != 0.0 || p.force[1] != 0.0 || p.force[2] != 0.0) ? 1 : 0;
}

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
    if (p.collision != LBM_SRT && p.collision != LBM_TRT) return LBM_ERR_ARG;
    if (p.storage < LBM_FP64 || p.storage > LBM_P16_1) return LBM_ERR_ARG;
    if (p.arith != LBM_ARITH_FP32 && p.arith != LBM_ARITH_FP64) return LBM_ERR_ARG;
    if (p.scheme != LBM_STREAM_AB && p.scheme != LBM_STREAM_AA) return LBM_ERR_ARG;
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

    const size_t fbytes = (size_t)h->q * N * h->sb;
    const int copies = h->aa() ? 1 : 2;
    for (int c = 0; c < copies; ++c) {
        h->f[c] = h->alloc(fbytes);
        if (!h->f[c]) { lbm_destroy(h); return LBM_ERR_OOM; }
    }
    h->scratch_doubles = std::max(kScratchDoubles, (size_t)h->plane() * std::max(h->q, 4));
    h->scratch_doubles = std::min(h->scratch_doubles, (size_t)std::max(h->q, 4) * N);
    h->partial = (double*)h->alloc((2 * kReduceBlocks + 2) * sizeof(double));
    if (!h->partial) { lbm_destroy(h); return LBM_ERR_OOM; }
    for (int c = 0; c < copies; ++c)
        if (h->cuda(cudaMemsetAsync(h->f[c], 0, fbytes, h->stream), "memset") != LBM_OK) {
            lbm_destroy(h);
            return LBM_ERR_CUDA;
        }
    *out = h;
    return LBM_OK;
}

extern "C" lbm_status lbm_destroy(lbm_handle* h) {
    if (!h) return LBM_OK;
    cudaStreamSynchronize(h->stream);
    for (void* ptr : h->allocations) h->al.release(ptr, h->al.ctx);
    h->allocations.clear();
    delete h;
    return LBM_OK;
}

extern "C" lbm_status lbm_set_block(lbm_handle* h, int bx, int by) {
    if (!h) return LBM_ERR_ARG;
    if (bx < 1 || by < 1 || bx * by > 256 || (bx * by) % 32 != 0) return h->fail(LBM_ERR_ARG, "block shape");
    h->bx = bx;
    h->by = by;
    return LBM_OK;
}

extern "C" lbm_status lbm_set_geometry(lbm_handle* h, const uint8_t* flags, const float* node_u, const float* node_rho) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    const size_t N = h->N;
    if (!flags) {
        h->release((void*&)h->flags, N);
        h->release((void*&)h->node_u, 3 * N * sizeof(float));
        h->release((void*&)h->node_rho, N * sizeof(float));
        return LBM_OK;
    }
    bool any_moving = false, any_eq = false;
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
        if (h->aa() && (fl & (LBM_OUTFLOW | LBM_FREESLIP)))
            return h->fail(LBM_ERR_UNSUPPORTED, "A-A streaming supports no OUTFLOW or FREESLIP cells");
        any_moving |= (fl & LBM_MOVING) != 0;
        any_eq |= (fl & LBM_EQ) != 0;
    }
    if (!h->flags) {
        h->flags = (uint8_t*)h->alloc(N);
        if (!h->flags) return h->fail(LBM_ERR_OOM, "flags");
    }
    if (h->cuda(cudaMemcpyAsync(h->flags, flags, N, cudaMemcpyHostToDevice, h->stream), "flags upload"))
        return LBM_ERR_CUDA;
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
            std::vector<float> ones(N, 1.0f);
            if (h->cuda(cudaMemcpyAsync(h->node_rho, ones.data(), N * sizeof(float), cudaMemcpyHostToDevice, h->stream),
                        "node_rho upload")) return LBM_ERR_CUDA;
            if (h->cuda(cudaStreamSynchronize(h->stream), "sync")) return LBM_ERR_CUDA;
        }
    }
    {
        const int grid = (int)std::min<size_t>((N + 255) / 256, 152 * 16);
        if (h->p.velset == LBM_D2Q9) k_mark_neighbours<D2Q9><<<grid, 256, 0, h->stream>>>(h->flags, h->p.nx, h->p.ny, h->p.nz);
        else if (h->p.velset == LBM_D3Q19) k_mark_neighbours<D3Q19><<<grid, 256, 0, h->stream>>>(h->flags, h->p.nx, h->p.ny, h->p.nz);
        else k_mark_neighbours<D3Q27><<<grid, 256, 0, h->stream>>>(h->flags, h->p.nx, h->p.ny, h->p.nz);
        if (h->cuda(cudaGetLastError(), "mark kernel")) return LBM_ERR_CUDA;
    }
    if (h->cuda(cudaStreamSynchronize(h->stream), "sync")) return LBM_ERR_CUDA;
    return LBM_OK;
}

namespace {

// zero every population copy and run the put kernel over z-chunks;
// `upload(z0, z1, dev)` stages the chunk's input doubles into dev
template <class R, class Up>
lbm_status put_all(lbm_handle* h, const Relax<R>& k, int setf, int per_cell, Up upload) {
    const size_t fbytes = (size_t)h->q * h->N * h->sb;
    for (int c = 0; c < (h->aa() ? 1 : 2); ++c)
        if (h->cuda(cudaMemsetAsync(h->f[c], 0, fbytes, h->stream), "memset")) return LBM_ERR_CUDA;
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
        if (h->cuda(h->ks->put[h->aa() ? 1 : 0](&pa, setf, L), "put kernel")) return LBM_ERR_CUDA;
        if (h->cuda(cudaStreamSynchronize(h->stream), "sync")) return LBM_ERR_CUDA;
    }
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

template <class R> lbm_status launch_one_step(lbm_handle* h, const Relax<R>& k, cudaStream_t s) {
    const int scheme = h->scheme_now();
    const StepArgs<R> a = h->args(k, h->aa() ? 0 : h->cur);
    const lbm_status st = h->cuda(h->ks->step[scheme][h->flags ? 1 : 0](&a, h->step_launch(s)), "step kernel");
    if (st != LBM_OK) return st;
    if (!h->aa()) h->cur ^= 1;
    h->t += 1;
    return LBM_OK;
}

}  // namespace

lbm_status lbm_internal_step(lbm_handle* h, cudaStream_t s) {
    return h->fp64() ? launch_one_step(h, h->kd, s) : launch_one_step(h, h->kf, s);
}

extern "C" lbm_status lbm_step(lbm_handle* h, int64_t nsteps) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    if (nsteps < 0) return h->fail(LBM_ERR_ARG, "negative step count");
    for (int64_t s = 0; s < nsteps; ++s) {
        st = lbm_internal_step(h, h->stream);
        if (st != LBM_OK) return st;
    }
    return LBM_OK;
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
    return LBM_OK;
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
        return h->cuda(cudaStreamSynchronize(h->stream), "sync");
    };
    return h->fp64() ? probe_chunks(h, h->kd, PROBE_FIELDS, 4, download)
                     : probe_chunks(h, h->kf, PROBE_FIELDS, 4, download);
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
        return h->cuda(cudaStreamSynchronize(h->stream), "sync");
    };
    return h->fp64() ? probe_chunks(h, h->kd, PROBE_F, h->q, download)
                     : probe_chunks(h, h->kf, PROBE_F, h->q, download);
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
    if (mass) *mass = res[0];
    if (energy) *energy = res[1];
    if (!std::isfinite(res[0]) || !std::isfinite(res[1])) return h->fail(LBM_ERR_DIVERGED, "non-finite mass or energy");
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_reduce(lbm_handle* h, double* mass, double* kinetic_energy) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    return h->fp64() ? reduce_impl(h, h->kd, mass, kinetic_energy) : reduce_impl(h, h->kf, mass, kinetic_energy);
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
    return LBM_OK;
}


extern "C" lbm_status lbm_autotune(lbm_handle* h, int trial_steps, int* bx_out, int* by_out) {
    lbm_status st = check_handle(h);
    if (st != LBM_OK) return st;
    if (trial_steps < 1) return h->fail(LBM_ERR_ARG, "trial_steps < 1");
    static const int shapes[][2] = {{128, 2}, {256, 1}, {64, 4}, {32, 8}, {64, 2}, {128, 1}, {32, 4}};
    cudaEvent_t ev[2];
    if (h->cuda(cudaEventCreate(&ev[0]), "event") || h->cuda(cudaEventCreate(&ev[1]), "event")) return LBM_ERR_CUDA;
    float best = 1e30f;
    int bb[2] = {h->bx, h->by};
    for (const auto& sh : shapes) {
        h->bx = sh[0];
        h->by = sh[1];
        if ((st = lbm_step(h, 2)) != LBM_OK) break;
        cudaEventRecord(ev[0], h->stream);
        if ((st = lbm_step(h, trial_steps)) != LBM_OK) break;
        cudaEventRecord(ev[1], h->stream);
        if (h->cuda(cudaEventSynchronize(ev[1]), "event sync")) { st = LBM_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (ms < best) { best = ms; bb[0] = sh[0]; bb[1] = sh[1]; }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    h->bx = bb[0];
    h->by = bb[1];
    if (bx_out) *bx_out = bb[0];
    if (by_out) *by_out = bb[1];
    return st;
}
