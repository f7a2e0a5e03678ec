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
using EnsFn = cudaError_t (*)(const void* members, const uint32_t* tile_member, int parity, const Launch&);
using ProbeFn = cudaError_t (*)(const void* probe_args, int mode, const Launch&);
using PutFn = cudaError_t (*)(const void* put_args, int setf, const Launch&);

struct KernelSet {
    StepFn step[3][2] = {};   // [scheme: AB, AA_PP, AA_LOC][flags]
    EnsFn ens[3] = {};        // [scheme], flags always on
    ProbeFn probe[3] = {};    // [layout: AB, AA swapped, AA natural]
    PutFn put[2] = {};        // [A-A]
    bool present = false;
};

// velset 0..2, collision 0..1, storage 0..9, arith 0 (FP32) / 1 (FP64)
KernelSet& kernel_set(int velset, int collision, int storage, int arith);

}  // namespace lbm
