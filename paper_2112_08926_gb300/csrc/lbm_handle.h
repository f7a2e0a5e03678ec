// Internal state of an lbm_handle, shared by the host units of the library.
#pragma once

#include <algorithm>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "lbm.h"
#include "lbm_kernels.cuh"
#include "lbm_registry.h"

using lbm::KernelSet;
using lbm::Launch;
using lbm::Relax;
using lbm::StepArgs;

struct lbm_handle {
    lbm_params p{};
    int q = 0;
    size_t N = 0;
    int sb = 0;
    lbm_allocator al{};
    cudaStream_t stream = nullptr;
    void* f[2] = {nullptr, nullptr};
    uint8_t* flags = nullptr;
    uint32_t* walls = nullptr;   // with flags: per-cell mask of the solid upstream directions (k_mark_neighbours)
    float* node_u = nullptr;
    float* node_rho = nullptr;
    double* scratch = nullptr;
    size_t scratch_doubles = 0;
    uint32_t* special = nullptr;   // cells that are not plain fluid (flagged lattices)
    uint32_t n_special = 0, special_cap = 0;
    uint32_t n_complex = 0;   // leading part of `special`: cells with rules beyond plain bounce-back
    bool has_open_boundaries = false;   // OUTFLOW or FREESLIP cells (A-B only)
    double* partial = nullptr;
    int64_t t = 0;
    int cur = 0;
    int64_t check_every = 0;   // lbm_set_divergence_check: steps between FP64 checks (0: off)
    double check_tol = 0.0, check_mass0 = 0.0;
    int bx = 128, by = 2;
    int variant = 0;           // requested stream-collide kernel variant (LBM_VARIANT_*)
    bool scheme_auto = false;  // created with LBM_STREAM_AUTO: lbm_autotune also picks the scheme
    int chunked = 0;           // populations in the chunked layout (16-bit storage, FP32 arithmetic)
    bool force_chunked = false;   // chunked whatever nx (set by an ensemble that steps its members so)
    int num_sms = 0;
    int* status = nullptr;     // device status word written by bounded waits
    lbm_status sticky = LBM_OK;
    std::string err;
    KernelSet* ks = nullptr;
    double* static_stage = nullptr;   // device address of the readback array of lbm_get_rho_u_static
    Relax<float> kf{};
    Relax<double> kd{};
    size_t device_bytes = 0;
    std::vector<void*> allocations;
    // CUDA graphs of kStepGraph consecutive steps, by (cur, t & 1) at their
    // start, captured on a private stream and replayed on `stream`; a graph
    // is valid while `gen` (bumped by every call that changes what a step
    // launches) equals the value it was captured at
    uint64_t gen = 0;
    uint64_t geom_gen = 0;     // bumped by lbm_set_geometry and lbm_set_nodes (cell lists, node values)
    cudaStream_t capture = nullptr;
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    uint64_t graph_gen[2][2] = {{0, 0}, {0, 0}};

    bool aa() const { return p.scheme == LBM_STREAM_AA; }
    // bytes of one population copy: 16-bit copies are padded to whole chunks
    // of 64 cells, so that the chunked layout fits any cell count
    size_t fbytes() const { return (size_t)q * (sb == 2 ? ((N + 63) & ~size_t(63)) : N) * sb; }
    // every population element index fits in 32 bits
    bool idx32() const { return (unsigned long long)q * N < (1ull << 32); }
    bool fp64() const { return p.arith == LBM_ARITH_FP64; }
    int plane() const { return p.nx * p.ny; }

    lbm_status fail(lbm_status s, const std::string& msg) {
        if (err.empty() || s == LBM_ERR_CUDA) err = msg;
        if (s == LBM_ERR_CUDA) sticky = s;
        return s;
    }
    lbm_status cuda(cudaError_t e, const char* what) {
        if (e == cudaSuccess) return LBM_OK;
        return fail(LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
    void* alloc(size_t bytes) {
        void* ptr = al.alloc(bytes, al.ctx);
        if (ptr) {
            allocations.push_back(ptr);
            device_bytes += bytes;
        }
        return ptr;
    }
    void release(void*& ptr, size_t bytes) {
        if (!ptr) return;
        for (size_t k = 0; k < allocations.size(); ++k)
            if (allocations[k] == ptr) { allocations.erase(allocations.begin() + k); break; }
        al.release(ptr, al.ctx);
        device_bytes -= bytes;
        ptr = nullptr;
    }

    // kernel argument block for the current state
    template <class R> StepArgs<R> args(const Relax<R>& k, int src_index) const {
        StepArgs<R> a{};
        a.src = f[src_index];
        a.dst = aa() ? f[0] : f[1 - src_index];
        a.flags = flags;
        a.walls = walls;
        a.node_u = node_u;
        a.node_rho = node_rho;
        a.nx = p.nx; a.ny = p.ny; a.nz = p.nz;
        a.N = (uint32_t)N;
        a.k = k;
        return a;
    }
    int scheme_now() const { return !aa() ? lbm::SCHEME_AB : ((t & 1) ? lbm::SCHEME_AA_LOC : lbm::SCHEME_AA_PP); }
    int layout_now() const {
        const int phase = !aa() ? lbm::LAYOUT_AB : ((t & 1) ? lbm::LAYOUT_AA_NATURAL : lbm::LAYOUT_AA_SWAPPED);
        return phase | (chunked ? lbm::LAYOUT_CHUNKED : 0);
    }
    Launch step_launch(cudaStream_t s) const {
        Launch L;
        L.block = dim3(bx, by, 1);
        L.grid = dim3((p.nx + bx - 1) / bx, (p.ny + by - 1) / by, p.nz);
        L.stream = s;
        return L;
    }
    int planes_per_chunk(int per_cell) const {
        size_t per_plane = (size_t)plane() * per_cell;
        size_t k = scratch_doubles / per_plane;
        return (int)std::max<size_t>(1, std::min<size_t>(k, (size_t)p.nz));
    }
};


// one stream-collide step of h launched on stream s (advances h's counters)
lbm_status lbm_internal_step(lbm_handle* h, cudaStream_t s);
// reads the device status word of h (after a stream synchronisation):
// LBM_ERR_TIMEOUT, and the handle poisoned, if a bounded wait gave up
lbm_status lbm_internal_check_status(lbm_handle* h);
// brings the stored populations into the layout the settings of h call for
// (after force_chunked changed)
lbm_status lbm_internal_ensure_layout(lbm_handle* h);
// device address of lbm_get_rho_u_static's staging array on the current
// device, looked up once per device; NULL if the look-up failed (the CUDA
// error is cleared)
double* lbm_internal_static_stage();
