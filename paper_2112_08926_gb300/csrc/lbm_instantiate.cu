// Instantiates every kernel for one storage format, arithmetic precision and
// velocity set.  The build compiles this file once per triple with
// -DLBM_FMT=<storage id> -DLBM_ARITH=<0 float | 1 double> -DLBM_VELSET=<0..2>,
// in parallel.
#include <type_traits>

#include "lbm_kernels.cuh"
#include "lbm_registry.h"

#ifndef LBM_FMT
#error "LBM_FMT must be defined"
#endif
#ifndef LBM_ARITH
#error "LBM_ARITH must be defined"
#endif
#ifndef LBM_VELSET
#error "LBM_VELSET must be defined (0 D2Q9, 1 D3Q19, 2 D3Q27)"
#endif

namespace lbm {
namespace {

using Real = std::conditional_t<LBM_ARITH == 1, double, float>;
constexpr int FMT = LBM_FMT;

template <class V, int COLL, int SCHEME, bool FLAGS, class IX, bool CH = false>
cudaError_t launch_step(const void* args, const Launch& L) {
    k_step<V, COLL, FMT, Real, SCHEME, FLAGS, IX, CH><<<L.grid, L.block, 0, L.stream>>>(
        *static_cast<const StepArgs<Real>*>(args));
    return cudaGetLastError();
}

template <class V, int COLL, int SCHEME, class IX, bool CH = false>
cudaError_t launch_list(const void* args, const uint32_t* cells, uint32_t count, const Launch& L) {
    k_step_list<V, COLL, FMT, Real, SCHEME, IX, CH><<<L.grid, L.block, 0, L.stream>>>(
        *static_cast<const StepArgs<Real>*>(args), cells, count);
    return cudaGetLastError();
}

template <class V, int COLL, int SCHEME, class IX, bool CH = false>
cudaError_t launch_ens(const void* members, const uint32_t* tile_member, int parity, const Launch& L) {
    k_ensemble_step<V, COLL, FMT, Real, SCHEME, IX, CH><<<L.grid, L.block, 0, L.stream>>>(
        static_cast<const EnsMember<Real>*>(members), tile_member, parity);
    return cudaGetLastError();
}

template <class V, int COLL, bool CH>
cudaError_t launch_ens_pair(const void* members, const uint32_t* tile_member, int parity, const Launch& L) {
    k_ensemble_pair<V, COLL, FMT, CH><<<L.grid, L.block, 0, L.stream>>>(
        static_cast<const EnsMember<float>*>(members), tile_member, parity);
    return cudaGetLastError();
}

template <class V, int COLL, int SCHEME, class IX, bool CH = false>
cudaError_t launch_ens_list(const void* members, const uint64_t* cells, uint32_t count, int parity, const Launch& L) {
    k_ensemble_list<V, COLL, FMT, Real, SCHEME, IX, CH><<<L.grid, L.block, 0, L.stream>>>(
        static_cast<const EnsMember<Real>*>(members), cells, count, parity);
    return cudaGetLastError();
}

template <class V, int LAYOUT>
cudaError_t launch_probe(const void* args, int mode, const Launch& L) {
    k_probe<V, FMT, Real, LAYOUT><<<L.grid, L.block, 0, L.stream>>>(
        *static_cast<const ProbeArgs<Real>*>(args), mode);
    return cudaGetLastError();
}

template <class V, int PL>
cudaError_t launch_put(const void* args, int setf, const Launch& L) {
    k_put<V, FMT, Real, PL><<<L.grid, L.block, 0, L.stream>>>(
        *static_cast<const PutArgs<Real>*>(args), setf);
    return cudaGetLastError();
}

template <class V, int COLL, int NX>
cudaError_t launch_staged(const void* args, int grid, int tiles_y, int* status, cudaStream_t stream) {
    constexpr int smem = StagedShape<NX, FMT>::template smem_bytes<V>();
    static bool configured = false;
    if (!configured) {
        const cudaError_t e = cudaFuncSetAttribute(k_step_staged<V, COLL, FMT, NX>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_step_staged<V, COLL, FMT, NX><<<grid, StagedShape<NX, FMT>::THREADS, smem, stream>>>(
        *static_cast<const StepArgs<float>*>(args), tiles_y, status);
    return cudaGetLastError();
}

template <class V, int COLL>
cudaError_t launch_pair(const void* args, const Launch& L) {
    k_step_pair<V, COLL, FMT><<<L.grid, L.block, 0, L.stream>>>(*static_cast<const StepArgs<float>*>(args));
    return cudaGetLastError();
}

template <class V, int COLL, int PHASE, bool PLAIN>
cudaError_t launch_pair_chunked(const void* args, const Launch& L) {
    k_step_pair_chunked<V, COLL, FMT, PHASE, PLAIN><<<L.grid, L.block, 0, L.stream>>>(
        *static_cast<const StepArgs<float>*>(args));
    return cudaGetLastError();
}

template <class V, int COLL>
void fill() {
    KernelSet& s = kernel_set(V::ID, COLL, FMT, LBM_ARITH);
    static_for<0, 3>([&](auto SC) {
        s.step[SC.value][0][0] = launch_step<V, COLL, SC.value, false, size_t>;
        s.step[SC.value][1][0] = launch_step<V, COLL, SC.value, true, size_t>;
        s.step[SC.value][0][1] = launch_step<V, COLL, SC.value, false, uint32_t>;
        s.step[SC.value][1][1] = launch_step<V, COLL, SC.value, true, uint32_t>;
        s.list[SC.value][0] = launch_list<V, COLL, SC.value, size_t>;
        s.list[SC.value][1] = launch_list<V, COLL, SC.value, uint32_t>;
        s.ens[SC.value][0] = launch_ens<V, COLL, SC.value, size_t>;
        s.ens[SC.value][1] = launch_ens<V, COLL, SC.value, uint32_t>;
        s.ens_list[SC.value][0] = launch_ens_list<V, COLL, SC.value, size_t>;
        s.ens_list[SC.value][1] = launch_ens_list<V, COLL, SC.value, uint32_t>;
    });
    s.probe[LAYOUT_AB] = launch_probe<V, LAYOUT_AB>;
    s.probe[LAYOUT_AA_SWAPPED] = launch_probe<V, LAYOUT_AA_SWAPPED>;
    s.probe[LAYOUT_AA_NATURAL] = launch_probe<V, LAYOUT_AA_NATURAL>;
    s.put[0] = launch_put<V, 0>;
    s.put[1] = launch_put<V, 1>;
    // the chunked layout and the paired kernels: 16-bit storage, FP32
    // arithmetic; D3Q27 only with the hardware conversions (FP16, FP16S: the
    // software codecs are bound by instruction issue, and the paired kernel
    // takes D3Q27's two cells one after the other to fit 27 code pairs)
    // MRT keeps the generic kernels (its 19 x 19 transforms per cell pair
    // would double the build for a kernel the operator cannot keep fed)
    if constexpr (LBM_ARITH == 0 && FMT >= 2 && COLL < 2 &&
                  (!std::is_same<V, D3Q27>::value || FMT == 2 || FMT == 3)) {
        s.probe[LAYOUT_AB_CHUNKED] = launch_probe<V, LAYOUT_AB_CHUNKED>;
        s.probe[LAYOUT_AA_SWAPPED_CHUNKED] = launch_probe<V, LAYOUT_AA_SWAPPED_CHUNKED>;
        s.probe[LAYOUT_AA_NATURAL_CHUNKED] = launch_probe<V, LAYOUT_AA_NATURAL_CHUNKED>;
        s.put[2] = launch_put<V, 2>;
        s.put[3] = launch_put<V, 3>;
        if constexpr (!std::is_same<V, D3Q27>::value) s.pair = launch_pair<V, COLL>;   // SoA paired: up to q = 19
        static_for<0, 3>([&](auto PH) {
            s.pair_chunked[PH.value][0] = launch_pair_chunked<V, COLL, PH.value, false>;
            s.pair_chunked[PH.value][1] = launch_pair_chunked<V, COLL, PH.value, true>;
            s.list_chunked[PH.value] = launch_list<V, COLL, PH.value, uint32_t, true>;
        });
    }
    // ensembles (D3Q19) of 16-bit members on the chunked layout, whatever
    // their nx: per-cell and generic single-lattice kernels with chunked
    // addressing; the paired ensemble kernel on both layouts (hardware
    // conversions only)
    if constexpr (LBM_ARITH == 0 && FMT >= 2 && COLL < 2 && std::is_same<V, D3Q19>::value) {
        static_for<0, 3>([&](auto SC) {
            s.step_ch[SC.value] = launch_step<V, COLL, SC.value, true, uint32_t, true>;
            s.ens_ch[SC.value] = launch_ens<V, COLL, SC.value, uint32_t, true>;
            s.ens_list_ch[SC.value] = launch_ens_list<V, COLL, SC.value, uint32_t, true>;
        });
        if constexpr (FMT == 2 || FMT == 3) {
            s.ens_pair[0] = launch_ens_pair<V, COLL, false>;
            s.ens_pair[1] = launch_ens_pair<V, COLL, true>;
        }
    }
    if constexpr (LBM_ARITH == 0 && FMT != 0 && COLL < 2 && std::is_same<V, D3Q19>::value) {
        s.staged[0] = launch_staged<V, COLL, 128>;
        s.staged[1] = launch_staged<V, COLL, 256>;
        s.staged[2] = launch_staged<V, COLL, 512>;
        s.staged_rows[0] = StagedShape<128, FMT>::H;
        s.staged_rows[1] = StagedShape<256, FMT>::H;
        s.staged_rows[2] = StagedShape<512, FMT>::H;
    }
    s.present = true;
}

struct Registrar {
    Registrar() {
        if constexpr (LBM_VELSET == 0) { fill<D2Q9, 0>(); fill<D2Q9, 1>(); }
        if constexpr (LBM_VELSET == 1) {
            fill<D3Q19, 0>();
            fill<D3Q19, 1>();
            // MRT for the storage formats of the paper's roofline comparison:
            // FP64 (FP64 arithmetic), FP32, FP16S and FP16C
            if constexpr ((FMT == 0 && LBM_ARITH == 1) || (LBM_ARITH == 0 && (FMT == 1 || FMT == 3 || FMT == 4)))
                fill<D3Q19, 2>();
        }
        if constexpr (LBM_VELSET == 2) { fill<D3Q27, 0>(); fill<D3Q27, 1>(); }
    }
};
const Registrar registrar;

}  // namespace
}  // namespace lbm
