// Instantiates every kernel for one storage format and arithmetic precision.
// The build compiles this file once per pair with -DLBM_FMT=<storage id>
// -DLBM_ARITH=<0 float | 1 double>, in parallel.
#include <type_traits>

#include "lbm_kernels.cuh"
#include "lbm_registry.h"

#ifndef LBM_FMT
#error "LBM_FMT must be defined"
#endif
#ifndef LBM_ARITH
#error "LBM_ARITH must be defined"
#endif

namespace lbm {
namespace {

using Real = std::conditional_t<LBM_ARITH == 1, double, float>;
constexpr int FMT = LBM_FMT;

template <class V, int COLL, int SCHEME, bool FLAGS>
cudaError_t launch_step(const void* args, const Launch& L) {
    k_step<V, COLL, FMT, Real, SCHEME, FLAGS><<<L.grid, L.block, 0, L.stream>>>(
        *static_cast<const StepArgs<Real>*>(args));
    return cudaGetLastError();
}

template <class V, int COLL, int SCHEME>
cudaError_t launch_ens(const void* members, const uint32_t* tile_member, int parity, const Launch& L) {
    k_ensemble_step<V, COLL, FMT, Real, SCHEME><<<L.grid, L.block, 0, L.stream>>>(
        static_cast<const EnsMember<Real>*>(members), tile_member, parity);
    return cudaGetLastError();
}

template <class V, int LAYOUT>
cudaError_t launch_probe(const void* args, int mode, const Launch& L) {
    k_probe<V, FMT, Real, LAYOUT><<<L.grid, L.block, 0, L.stream>>>(
        *static_cast<const ProbeArgs<Real>*>(args), mode);
    return cudaGetLastError();
}

template <class V, bool AA>
cudaError_t launch_put(const void* args, int setf, const Launch& L) {
    k_put<V, FMT, Real, AA><<<L.grid, L.block, 0, L.stream>>>(
        *static_cast<const PutArgs<Real>*>(args), setf);
    return cudaGetLastError();
}

template <class V, int COLL>
void fill() {
    KernelSet& s = kernel_set(V::ID, COLL, FMT, LBM_ARITH);
    s.step[SCHEME_AB][0] = launch_step<V, COLL, SCHEME_AB, false>;
    s.step[SCHEME_AB][1] = launch_step<V, COLL, SCHEME_AB, true>;
    s.step[SCHEME_AA_PP][0] = launch_step<V, COLL, SCHEME_AA_PP, false>;
    s.step[SCHEME_AA_PP][1] = launch_step<V, COLL, SCHEME_AA_PP, true>;
    s.step[SCHEME_AA_LOC][0] = launch_step<V, COLL, SCHEME_AA_LOC, false>;
    s.step[SCHEME_AA_LOC][1] = launch_step<V, COLL, SCHEME_AA_LOC, true>;
    s.ens[SCHEME_AB] = launch_ens<V, COLL, SCHEME_AB>;
    s.ens[SCHEME_AA_PP] = launch_ens<V, COLL, SCHEME_AA_PP>;
    s.ens[SCHEME_AA_LOC] = launch_ens<V, COLL, SCHEME_AA_LOC>;
    s.probe[LAYOUT_AB] = launch_probe<V, LAYOUT_AB>;
    s.probe[LAYOUT_AA_SWAPPED] = launch_probe<V, LAYOUT_AA_SWAPPED>;
    s.probe[LAYOUT_AA_NATURAL] = launch_probe<V, LAYOUT_AA_NATURAL>;
    s.put[0] = launch_put<V, false>;
    s.put[1] = launch_put<V, true>;
    s.present = true;
}

struct Registrar {
    Registrar() {
        fill<D2Q9, 0>(); fill<D2Q9, 1>();
        fill<D3Q19, 0>(); fill<D3Q19, 1>();
        fill<D3Q27, 0>(); fill<D3Q27, 1>();
    }
};
const Registrar registrar;

}  // namespace
}  // namespace lbm
