// Type-erased launchers of the templated kernels, one table per
// (velocity set, collision, storage format, arithmetic precision).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

struct Launch {
    dim3 grid, block;
    cudaStream_t stream;
};

using StepFn = cudaError_t (*)(const void* step_args, const Launch&);
// cells of a flagged lattice from a list (see k_step_list)
using ListFn = cudaError_t (*)(const void* step_args, const uint32_t* cells, uint32_t count, const Launch&);
using EnsFn = cudaError_t (*)(const void* members, const uint32_t* tile_member, int parity, const Launch&);
using EnsListFn = cudaError_t (*)(const void* members, const uint64_t* cells, uint32_t count, int parity,
                                  const Launch&);
using ProbeFn = cudaError_t (*)(const void* probe_args, int mode, const Launch&);
using PutFn = cudaError_t (*)(const void* put_args, int setf, const Launch&);
// staged flag-free A-B step: grid size, tiles along y, status word
using StagedFn = cudaError_t (*)(const void* step_args, int grid, int tiles_y, int* status, cudaStream_t);

struct KernelSet {
    StepFn step[3][2][2] = {};   // [scheme: AB, AA_PP, AA_LOC][flags][32-bit indices]
    ListFn list[3][2] = {};      // [scheme][32-bit indices]: the non-plain cells of a flagged lattice
    ListFn list_chunked[3] = {}; // [scheme]: the same on the chunked layout
    StepFn step_ch[3] = {};      // [scheme]: generic kernel, chunked addressing, flags, 32-bit indices (D3Q19)
    EnsFn ens[3][2] = {};        // [scheme][32-bit indices], flags always on: plain cells
    EnsListFn ens_list[3][2] = {};   // the listed non-plain cells of all members
    EnsFn ens_pair[2] = {};      // paired ensemble step [chunked layout] (A-B, 32-bit indices, FP16 / FP16S, D3Q19)
    EnsFn ens_ch[3] = {};        // [scheme]: per-cell ensemble step on the chunked layout (32-bit indices)
    EnsListFn ens_list_ch[3] = {};   // [scheme]: the listed cells on the chunked layout
    ProbeFn probe[8] = {};    // [layout code: phase | 4 if chunked]
    PutFn put[4] = {};        // [bit 0: A-A, bit 1: chunked]
    StagedFn staged[3] = {};  // row length 128, 256, 512 (D3Q19, FP32 arithmetic only)
    int staged_rows[3] = {};  // rows per tile
    StepFn pair = nullptr;    // two cells per thread (flag-free A-B, 16-bit storage)
    StepFn pair_chunked[3][2] = {};  // chunked layout: [phase: A-B, A-A odd, A-A even][plain cells only]
    bool present = false;
};

// velset 0..2, collision 0..2 (MRT: D3Q19), storage 0..9, arith 0 (FP32) / 1 (FP64)
KernelSet& kernel_set(int velset, int collision, int storage, int arith);

}  // namespace lbm
