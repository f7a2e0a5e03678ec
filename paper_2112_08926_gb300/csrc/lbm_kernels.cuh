// Stream-collide kernels for sm_103a (arXiv 2112.08926, appendix "LBM
// equations in a nutshell" with DDF shifting, fused into one pass per step).
//
// One thread updates one cell; consecutive threads take consecutive x, so
// every population array is read and written with coalesced warp accesses in
// structure-of-arrays order f[i*N + n].  Neighbour indices come from three
// wrapped offsets per axis (no integer division in the loop).  Streaming
// schemes:
//   AB     pull from copy A, write copy B (the paper's one-step pull, Sec. 5);
//   AA_PP  in-place, odd half of A-A: pull each population from the
//          opposite slot of the upstream cell, push the result into the
//          downstream cell's slot;
//   AA_LOC in-place, even half: read the own slots, write the opposite ones.
// Both A-A halves touch exactly the memory they read, so one copy suffices,
// and they give bit-for-bit the A-B result.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

enum { SCHEME_AB = 0, SCHEME_AA_PP = 1, SCHEME_AA_LOC = 2 };
// Memory layouts: the phase of the streaming scheme (A-B, or the A-A slots
// before an odd or an even step) in the low bits, LAYOUT_CHUNKED as a flag.
enum {
    LAYOUT_AB = 0, LAYOUT_AA_SWAPPED = 1, LAYOUT_AA_NATURAL = 2, LAYOUT_CHUNKED = 4,
    LAYOUT_AB_CHUNKED = 4, LAYOUT_AA_SWAPPED_CHUNKED = 5, LAYOUT_AA_NATURAL_CHUNKED = 6
};
constexpr int layout_phase(int layout) { return layout & 3; }
constexpr bool layout_chunked(int layout) { return (layout & LAYOUT_CHUNKED) != 0; }

// Chunked (array-of-structure-of-arrays) layout of a 16-bit lattice with nx
// a multiple of 64: the cells of a row are cut into chunks of 64 consecutive
// x; chunk c = n / 64 stores its q populations (slots) one after the other,
// 64 codes each.  Element of slot i of cell n:
constexpr int CHUNK = 64;
template <class V>
__host__ __device__ __forceinline__ size_t chunk_elem(int i, uint32_t n) {
    return ((size_t)(n >> 6) * (size_t)V::Q + (size_t)i) * CHUNK + (n & (CHUNK - 1));
}
enum { PROBE_FIELDS = 0, PROBE_F = 1, PROBE_REDUCE = 2 };

// internal flag bits of non-solid cells, set by the library after upload:
// a neighbour is solid (or the cell is an outflow cell), a neighbour is a
// free-slip wall, a neighbour is a moving wall.  A cell whose byte is
// F_NEAR_SOLID alone needs plain bounce-back only (no moving, free-slip,
// equilibrium or outflow rule): the fast kernels update it themselves.
constexpr uint32_t F_NEAR_SOLID = 0x20u;
constexpr uint32_t F_NEAR_FREESLIP = 0x40u;
constexpr uint32_t F_NEAR_MOVING = 0x80u;

template <class R> struct StepArgs {
    const void* src;          // A-B: copy read this step; A-A: the single copy
    void* dst;                // A-B: copy written; A-A: same as src
    const uint8_t* flags;     // NULL for the flag-free periodic kernel
    const uint32_t* walls;    // with flags: bit i of cell n set if the upstream cell n - c_i is solid
    const float* node_u;      // 3*N, component-major
    const float* node_rho;    // N
    int nx, ny, nz;
    uint32_t N;
    Relax<R> k;
    int pf;                   // L2 prefetch distance: z-planes (chunked kernels), tiles (ensemble); 0: none
    int pf_y;                 // chunked kernels: further rows of the prefetch distance (< ny)
};

struct Nbr {
    uint32_t xo[3], yo[3], zo[3];   // wrapped offsets for delta = -1, 0, +1
    __device__ __forceinline__ Nbr(int x, int y, int z, int nx, int ny, int nz) {
        const uint32_t plane = (uint32_t)nx * (uint32_t)ny;
        xo[0] = x == 0 ? nx - 1 : x - 1;
        xo[1] = x;
        xo[2] = x == nx - 1 ? 0 : x + 1;
        yo[0] = (uint32_t)(y == 0 ? ny - 1 : y - 1) * nx;
        yo[1] = (uint32_t)y * nx;
        yo[2] = (uint32_t)(y == ny - 1 ? 0 : y + 1) * nx;
        zo[0] = (uint32_t)(z == 0 ? nz - 1 : z - 1) * plane;
        zo[1] = (uint32_t)z * plane;
        zo[2] = (uint32_t)(z == nz - 1 ? 0 : z + 1) * plane;
    }
    // cell x - c_i (upstream) and x + c_i (downstream)
    template <class V, int I> __device__ __forceinline__ uint32_t up() const {
        return xo[1 - V::c(I, 0)] + yo[1 - V::c(I, 1)] + zo[1 - V::c(I, 2)];
    }
    template <class V, int I> __device__ __forceinline__ uint32_t down() const {
        return xo[1 + V::c(I, 0)] + yo[1 + V::c(I, 1)] + zo[1 + V::c(I, 2)];
    }
    __device__ __forceinline__ uint32_t self() const { return xo[1] + yo[1] + zo[1]; }
};

// Address of element j of population slot `slot` in a population-major
// copy.  With 32-bit indices (q N < 2^32) the element offset is one 32-bit
// multiply-add; otherwise the slot's start (a product of kernel arguments
// only, kept in uniform registers) is added to the 32-bit cell index, so
// 64-bit lattices pay no 64-bit index arithmetic per thread.
// On the chunked layout (CH) the element is chunk_elem.
template <class IX, bool CH, class V, class T>
__device__ __forceinline__ T* elem_ptr(T* p, int slot, uint32_t N, uint32_t j) {
    if constexpr (CH) return p + chunk_elem<V>(slot, j);
    else if constexpr (sizeof(IX) == 4) return p + ((uint32_t)slot * N + j);
    else return (p + (size_t)slot * (size_t)N) + j;
}

// Moving-wall term of the bounce-back (Sec. 4.4): 6 w_i rho_w (c_i . u_w),
// rho_w = 1, u_w read at the wall cell m.
template <class V, int I, class R, int SL>
__device__ __forceinline__ R moving_term(const float* node_u, size_t N, uint32_t m) {
    const R uw[3] = {(R)node_u[m], (R)node_u[N + m], (R)node_u[2 * N + m]};
    return R(6.0 * V::w(I) * Pow2<SL>::up) * csum<V, I, R>(uw);
}

// Streamed populations of a cell next to solid cells (or an outflow cell),
// streaming at `nb`.  A solid upstream cell reflects the cell's own opposite
// population (mid-grid bounce-back, Sec. 4.1), plus the moving-wall term; a
// free-slip upstream cell (A-B only) hands over the mirror population of the
// cell beside it, or bounce-back if that cell is solid too.  Addresses are
// chosen with selects and all loads are issued before the moving-wall terms
// are added, so the loads stay in flight together.
// Returns the mask of directions whose upstream cell is solid (bit i).
template <class V, int FMT, class R, bool AA, class IX, bool CH>
__device__ __forceinline__ uint32_t gather_boundary(const StepArgs<R>& a, const typename Storage<FMT>::T* src,
                                                    const Nbr& nb, R* f) {
    using S = Storage<FMT>;
    const uint32_t N = a.N;
    const uint32_t self = nb.self();
    uint32_t fy[V::Q];
    static_for<0, V::Q>([&](auto I) { fy[I.value] = a.flags[nb.up<V, I.value>()]; });
    static_for<0, V::Q>([&](auto I) {
        constexpr int i = I.value;
        constexpr int slot = AA ? opposite(i) : i;
        constexpr int bslot = AA ? i : opposite(i);
        const uint32_t j = nb.up<V, i>();
        const bool wall = fy[i] & F_WALL;
        int sl = wall ? bslot : slot;          // source population and cell
        uint32_t cell = wall ? self : j;
        if constexpr (!AA) {
            constexpr int cx = V::c(i, 0), cy = V::c(i, 1), cz = V::c(i, 2);
            constexpr int m0 = mirror<V>(i, 0), m1 = mirror<V>(i, 1), m2 = mirror<V>(i, 2);
            const uint32_t axis = (fy[i] >> 5) & 3u;
            const bool fs = wall && (fy[i] & F_FREESLIP) && axis < 3u;
            // compile-time array indices only (a runtime index would put nb in local memory)
            const uint32_t j2 = (axis == 0 ? nb.xo[1] : nb.xo[1 - cx]) + (axis == 1 ? nb.yo[1] : nb.yo[1 - cy]) +
                                (axis == 2 ? nb.zo[1] : nb.zo[1 - cz]);
            const uint32_t f2 = fs ? (uint32_t)a.flags[j2] : F_WALL;
            if (!(f2 & F_WALL)) {
                sl = axis == 0 ? m0 : (axis == 1 ? m1 : m2);
                cell = j2;
            }
        }
        f[i] = S::template load_g<R>(elem_ptr<IX, CH, V>(src, sl, N, cell), 0u);
    });
    uint32_t walls = 0;
    static_for<0, V::Q>([&](auto I) {
        constexpr int i = I.value;
        if (fy[i] & F_MOVING) f[i] = f[i] + moving_term<V, i, R, S::SL>(a.node_u, a.N, nb.up<V, i>());
        walls |= (fy[i] & F_WALL) ? (1u << i) : 0u;
    });
    return walls;
}

// Streamed populations of cell n at (x,y,z) for the given memory layout.
// Cells without solid neighbours (internal bit F_NEAR_SOLID clear) take the
// plain pull, as in the flag-free kernel.
// Returns the solid-upstream mask of gather_boundary (0 on the other paths).
template <class V, int FMT, class R, bool FLAGS, int LAYOUT, class IX = size_t>
__device__ __forceinline__ uint32_t gather(const StepArgs<R>& a, const typename Storage<FMT>::T* src,
                                           int x, int y, int z, uint32_t n, uint32_t fl, R* f) {
    using S = Storage<FMT>;
    constexpr int PH = layout_phase(LAYOUT);
    constexpr bool CH = layout_chunked(LAYOUT);
    if constexpr (PH == LAYOUT_AA_NATURAL) {
        static_for<0, V::Q>([&](auto I) {
            f[I.value] = S::template load_g<R>(elem_ptr<IX, CH, V>(src, I.value, a.N, n), 0u);
        });
        if (FLAGS && (fl & F_NEAR_MOVING)) {
            const Nbr nb(x, y, z, a.nx, a.ny, a.nz);
            static_for<1, V::Q>([&](auto I) {
                const uint32_t j = nb.up<V, I.value>();
                if (a.flags[j] & F_MOVING) f[I.value] = f[I.value] + moving_term<V, I.value, R, S::SL>(a.node_u, a.N, j);
            });
        }
    } else {
        constexpr bool AA = PH == LAYOUT_AA_SWAPPED;
        if (FLAGS && (fl & F_NEAR_SOLID)) {
            int sx = x;
            if (!AA && (fl & F_OUTFLOW)) sx = x == 0 ? a.nx - 1 : x - 1;
            const Nbr nb(sx, y, z, a.nx, a.ny, a.nz);
            return gather_boundary<V, FMT, R, AA, IX, CH>(a, src, nb, f);
        } else {
            const Nbr nb(x, y, z, a.nx, a.ny, a.nz);
            static_for<0, V::Q>([&](auto I) {
                constexpr int slot = AA ? opposite(I.value) : I.value;
                f[I.value] = S::template load_g<R>(elem_ptr<IX, CH, V>(src, slot, a.N, nb.up<V, I.value>()), 0u);
            });
        }
    }
    return 0u;
}

// One fused stream-collide update of cell (x, y, z).  PLAIN_ONLY (with
// flags): only cells whose flag byte is 0 -- fluid, no solid, moving or
// equilibrium neighbour -- are updated; the others are left to the list
// kernel, so no warp runs the boundary path for a few of its lanes.
template <class V, int COLL, int FMT, class R, int SCHEME, bool FLAGS, class IX, bool PLAIN_ONLY = false,
          bool CH = false, bool SPEC = true>
__device__ __forceinline__ void cell_step(const StepArgs<R>& a, int x, int y, int z) {
    using S = Storage<FMT>;
    using T = typename S::T;
    const uint32_t n = (uint32_t)x + (uint32_t)a.nx * ((uint32_t)y + (uint32_t)a.ny * (uint32_t)z);
    const T* src = (const T*)a.src;
    T* dst = (T*)a.dst;
    constexpr int PH = SCHEME == SCHEME_AB ? LAYOUT_AB
                     : (SCHEME == SCHEME_AA_PP ? LAYOUT_AA_SWAPPED : LAYOUT_AA_NATURAL);
    constexpr int LAYOUT = PH | (CH ? LAYOUT_CHUNKED : 0);
    // PLAIN_ONLY reads the flag byte too, but compiles no boundary code
    const uint32_t fl = (FLAGS || PLAIN_ONLY) ? (uint32_t)a.flags[n] : 0u;
    // SPEC: the plain pull is issued for every cell together with the flag
    // load, so the two memory latencies overlap; solid and equilibrium cells
    // drop it, cells next to solid cells gather again with their boundaries.
    // Without SPEC (cells known to be boundary cells) each cell gathers once.
    R f[V::Q];
    uint32_t walls = 0;   // directions with a solid upstream (= downstream of the opposite) cell
    if constexpr (SPEC) gather<V, FMT, R, false, LAYOUT, IX>(a, src, x, y, z, n, 0u, f);
    if (PLAIN_ONLY && fl != 0u) {
        // plain bounce-back cells stay: a direction whose upstream cell is
        // solid takes the cell's own opposite population instead, as in
        // gather_boundary (the even A-A half reads own slots only and has
        // nothing to replace); every other non-plain cell is listed
        if (fl != F_NEAR_SOLID) return;
        if constexpr (PH != LAYOUT_AA_NATURAL) {
            // the wall mask of the cell, then its own populations of the
            // bounce-back directions
            walls = a.walls[n];
            static_for<1, V::Q>([&](auto I) {
                constexpr int i = I.value;
                constexpr int bslot = PH == LAYOUT_AA_SWAPPED ? i : opposite(i);
                if ((walls >> i) & 1u) f[i] = S::template load_g<R>(elem_ptr<IX, CH, V>(src, bslot, a.N, n), 0u);
            });
        }
    }
    if (FLAGS && (fl & F_WALL)) return;
    if (FLAGS && (fl & F_EQ)) {
        const R u[3] = {(R)a.node_u[n], (R)a.node_u[(size_t)a.N + n], (R)a.node_u[2 * (size_t)a.N + n]};
        equilibrium_only<V, R, S::SL>((R)a.node_rho[n], u, f, a.k.sh);
    } else {
        if constexpr (!SPEC)
            walls = gather<V, FMT, R, FLAGS, LAYOUT, IX>(a, src, x, y, z, n, fl, f);
        else if (FLAGS && (fl & (PH == LAYOUT_AA_NATURAL ? F_NEAR_MOVING : F_NEAR_SOLID)))
            walls = gather<V, FMT, R, true, LAYOUT, IX>(a, src, x, y, z, n, fl, f);
        collide<V, COLL, R, S::SL, (FMT >= 2)>(a.k, f);
    }
    if constexpr (SCHEME == SCHEME_AB) {
        static_for<0, V::Q>([&](auto I) { S::template store_g<R>(elem_ptr<IX, CH, V>(dst, I.value, a.N, n), 0u, f[I.value]); });
    } else if constexpr (SCHEME == SCHEME_AA_LOC) {
        static_for<0, V::Q>([&](auto I) {
            S::template store_g<R>(elem_ptr<IX, CH, V>(dst, opposite(I.value), a.N, n), 0u, f[I.value]);
        });
    } else {
        const Nbr nb(x, y, z, a.nx, a.ny, a.nz);
        if ((FLAGS || PLAIN_ONLY) && (fl & F_NEAR_SOLID)) {
            static_for<0, V::Q>([&](auto I) {
                constexpr int i = I.value;
                const uint32_t d = nb.down<V, i>();
                // the downstream cell of i is the upstream cell of opposite(i)
                const bool wall = (walls >> opposite(i)) & 1u;   // reflected back into this cell
                S::template store_g<R>(elem_ptr<IX, CH, V>(dst, wall ? opposite(i) : i, a.N, wall ? n : d), 0u, f[i]);
            });
        } else {
            static_for<0, V::Q>([&](auto I) {
                S::template store_g<R>(elem_ptr<IX, CH, V>(dst, I.value, a.N, nb.down<V, I.value>()), 0u, f[I.value]);
            });
        }
    }
}

// IX: element-index type, uint32_t when q*N < 2^32 (cheaper address arithmetic).
// MRT's two 19 x 19 transforms need about 80 registers: 3 blocks per SM
// instead of 4 keep them without spills.
// FLAGS: the lattice has flags; then this kernel updates the plain cells
// (flag byte 0) only and k_step_list the listed others.
// CH: populations on the chunked layout (any nx; used for the members of an
// ensemble that steps them on that layout).
template <class V, int COLL, int FMT, class R, int SCHEME, bool FLAGS, class IX, bool CH = false>
__global__ void __launch_bounds__(256, (sizeof(R) == 8 || (SCHEME == SCHEME_AA_PP && sizeof(IX) == 8)) ? 2 : (COLL == 2 ? 3 : 4))
    k_step(const StepArgs<R> a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    // with flags: the flag-free update of the plain cells only (no boundary code)
    cell_step<V, COLL, FMT, R, SCHEME, false, IX, FLAGS, CH>(a, x, y, (int)blockIdx.z);
}

// The non-plain cells of a flagged lattice (solid cells excluded): boundary
// neighbours, equilibrium and outflow cells, from a list built when the
// geometry is set, one per thread.
template <class V, int COLL, int FMT, class R, int SCHEME, class IX, bool CH>
__global__ void __launch_bounds__(256, (SCHEME == SCHEME_AA_PP && sizeof(IX) == 8) ? 2 : 3)
    k_step_list(const StepArgs<R> a, const uint32_t* __restrict__ cells, uint32_t count) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const uint32_t n = cells[t];
    const uint32_t plane = (uint32_t)a.nx * (uint32_t)a.ny;
    const uint32_t z = n / plane, r = n - z * plane;
    const uint32_t y = r / (uint32_t)a.nx, x = r - y * (uint32_t)a.nx;
    cell_step<V, COLL, FMT, R, SCHEME, true, IX, false, CH, false>(a, (int)x, (int)y, (int)z);
}

// ---------------------------------------------------------------- staged kernel
// Flag-free periodic A-B step with the source rows staged in shared memory by
// the bulk-copy engine.  A persistent CTA of NX*H threads walks tiles of H
// whole x-rows (one z-plane); for every tile, warp 0 issues one
// cp.async.bulk per (population, row) -- the row (y - c_y, z - c_z) of
// population i, exactly the cells that stream into the tile -- completing on
// the stage's mbarrier.  STAGES tiles are in flight while one is computed,
// so the bytes in flight do not depend on registers.  Each population load
// is then one shared-memory read at a constant offset (x-wrap by selecting
// x-1, x or x+1); the per-cell arithmetic is cell_step's.  Every wait is
// bounded: on timeout the CTA writes *status = 1, waits (bounded) for the
// copies it still has in flight and returns.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    // suspends for at most ~2 us per poll (time-limit hint in ns)
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity), "r"(2000u) : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait: gives up after about a second (global timer), or after 2^24
// polls should the timer not advance
constexpr uint64_t kWaitLimitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    for (uint32_t k = 0; k < (1u << 24); ++k) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((k & 63) == 63 && global_ns() - t0 > kWaitLimitNs) return false;
    }
    return false;
}

template <int NX, int FMT> struct StagedShape {
    using T = typename Storage<FMT>::T;
    static constexpr int THREADS = 512;
    static constexpr int H = THREADS / NX;              // rows per tile
    static constexpr int ROW = NX * (int)sizeof(T);     // bytes per staged row
    static constexpr int STAGES = sizeof(T) == 2 ? 3 : 2;
    template <class V> static constexpr int stage_bytes() { return V::Q * H * ROW; }
    template <class V> static constexpr int smem_bytes() { return STAGES * stage_bytes<V>() + 8 * STAGES; }
};

template <class V, int COLL, int FMT, int NX>
__global__ void __launch_bounds__(512, 2) k_step_staged(const StepArgs<float> a, int tiles_y, int* status) {
    using S = Storage<FMT>;
    using T = typename S::T;
    using Sh = StagedShape<NX, FMT>;
    constexpr int H = Sh::H, ROW = Sh::ROW, STAGES = Sh::STAGES;
    constexpr int STAGE_BYTES = Sh::template stage_bytes<V>();
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x = tid % NX, r = tid / NX;
    const int ntiles = tiles_y * a.nz;
    if ((int)blockIdx.x >= ntiles) return;
    const int my = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    const uint32_t N = a.N;
    const uint32_t plane = (uint32_t)NX * (uint32_t)a.ny;
    if (tid == 0) {
        for (int st = 0; st < STAGES; ++st) mbar_init(&bars[st], 1);
        mbar_fence_init();
    }
    __syncthreads();

    // warp 0 (all lanes compute the same addresses, lane 0 issues): stage tile k into buffer st
    auto issue = [&](int k, int st) {
        const int t = (int)blockIdx.x + k * (int)gridDim.x;
        const int z = t / tiles_y, y0 = (t - z * tiles_y) * H;
        if (lane == 0) mbar_expect_tx(&bars[st], STAGE_BYTES);
        unsigned char* base = smem + st * STAGE_BYTES;
        static_for<0, V::Q>([&](auto I) {
            constexpr int i = I.value, cy = V::c(i, 1), cz = V::c(i, 2);
            const int zs = z - cz < 0 ? a.nz - 1 : (z - cz >= a.nz ? 0 : z - cz);
#pragma unroll
            for (int rr = 0; rr < H; ++rr) {
                // rows of a ragged last tile may lie past ny: any in-range row will do
                int ys = y0 + rr - cy;
                if (ys < 0) ys += a.ny;
                while (ys >= a.ny) ys -= a.ny;
                const T* src = (const T*)a.src + (i * N + (uint32_t)zs * plane + (uint32_t)ys * NX);
                if (lane == 0) bulk_g2s(base + (i * H + rr) * ROW, src, ROW, &bars[st]);
            }
        });
    };

    if (warp == 0)
        for (int k = 0; k < STAGES && k < my; ++k) issue(k, k);
    const int xm = x == 0 ? NX - 1 : x - 1, xp = x == NX - 1 ? 0 : x + 1;
    T* dst = (T*)a.dst;
    for (int k = 0; k < my; ++k) {
        const int st = k % STAGES;
        const bool ok = mbar_wait(&bars[st], (uint32_t)((k / STAGES) & 1));
        if (__syncthreads_or(!ok)) {   // CTA-uniform: flag, let the copies in flight land, leave
            if (tid == 0) {
                atomicExch(status, 1);
                for (int q = k; q < my && q < k + STAGES; ++q) mbar_wait(&bars[q % STAGES], (uint32_t)((q / STAGES) & 1));
            }
            return;
        }
        const int t = (int)blockIdx.x + k * (int)gridDim.x;
        const int z = t / tiles_y, y = (t - z * tiles_y) * H + r;
        if (y < a.ny) {
            const T* tile = (const T*)(smem + st * STAGE_BYTES) + r * NX;
            float f[V::Q];
            static_for<0, V::Q>([&](auto I) {
                constexpr int i = I.value, cx = V::c(i, 0);
                const int xs = cx == 0 ? x : (cx > 0 ? xm : xp);
                f[i] = S::template load_g<float>(tile, (uint32_t)(i * H * NX + xs));
            });
            collide<V, COLL, float, S::SL, (FMT >= 2)>(a.k, f);
            const uint32_t n = (uint32_t)z * plane + (uint32_t)y * NX + x;
            static_for<0, V::Q>([&](auto I) { S::template store_g<float>(dst, (uint32_t)I.value * N + n, f[I.value]); });
        }
        __syncthreads();
        if (warp == 0 && k + STAGES < my) issue(k + STAGES, st);
    }
}

// ---------------------------------------------------------------- paired kernel
// Flag-free periodic A-B step for 16-bit storage with two x-neighbouring
// cells per thread: every population is read and written as one 32-bit pair
// of codes.  A pair shifted by one cell in x (c_x != 0) is assembled from the
// thread's own aligned pair and the neighbouring lane's (warp shuffle); at the
// end of a warp and at the periodic wrap the missing code is read directly.
// Needs nx even, q*N < 2^32 and a block width that is a multiple of 32 (a warp
// then covers one row segment).  Per-cell arithmetic is cell_step's.
template <class V, int COLL, int FMT>
__global__ void __launch_bounds__(256, 3) k_step_pair(const StepArgs<float> a) {
    using C = Codec16<FMT>;
    constexpr int SL = C::SL;
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const int lane = threadIdx.x & 31;
    const bool active = (2 * px < a.nx) && (y < a.ny);
    // inactive threads stay for the shuffles, reading a valid pair
    const int x0 = active ? 2 * px : 0;
    const int yc = y < a.ny ? y : 0;
    const uint32_t nx = (uint32_t)a.nx, plane = nx * (uint32_t)a.ny, N = a.N;
    const uint32_t yo[3] = {(uint32_t)(yc == 0 ? a.ny - 1 : yc - 1) * nx, (uint32_t)yc * nx,
                            (uint32_t)(yc == a.ny - 1 ? 0 : yc + 1) * nx};
    const uint32_t zo[3] = {(uint32_t)(z == 0 ? a.nz - 1 : z - 1) * plane, (uint32_t)z * plane,
                            (uint32_t)(z == a.nz - 1 ? 0 : z + 1) * plane};
    const uint32_t xm = x0 == 0 ? nx - 1 : (uint32_t)x0 - 1;        // source of x0 when c_x = +1
    const uint32_t xp2 = (uint32_t)x0 + 2 == nx ? 0 : (uint32_t)x0 + 2; // source of x0+1 when c_x = -1
    const bool edge_lo = lane == 0 || x0 == 0;
    const bool edge_hi = lane == 31 || (uint32_t)x0 + 2 == nx;
    const uint16_t* src = (const uint16_t*)a.src;
    uint32_t g[V::Q];   // lo half: cell x0, hi half: cell x0 + 1
    static_for<0, V::Q>([&](auto I) {
        constexpr int i = I.value, cx = V::c(i, 0), cy = V::c(i, 1), cz = V::c(i, 2);
        const uint32_t row = (uint32_t)i * N + yo[1 - cy] + zo[1 - cz];
        const uint32_t P = *reinterpret_cast<const uint32_t*>(src + row + (uint32_t)x0);
        if constexpr (cx == 0) {
            g[i] = P;
        } else if constexpr (cx > 0) {      // sources x0-1, x0
            const uint32_t Pu = __shfl_up_sync(0xffffffffu, P, 1);
            const uint32_t e = edge_lo ? (uint32_t)src[row + xm] : (Pu >> 16);
            g[i] = (P << 16) | e;
        } else {                            // sources x0+1, x0+2
            const uint32_t Pd = __shfl_down_sync(0xffffffffu, P, 1);
            const uint32_t e = edge_hi ? (uint32_t)src[row + xp2] : (Pd & 0xFFFFu);
            g[i] = (P >> 16) | (e << 16);
        }
    });
    float f[V::Q];
    if constexpr (FMT == 2 || FMT == 3) {   // hardware conversions: both cells at once
        float fb[V::Q];
        static_for<0, V::Q>([&](auto I) {
            f[I.value] = C::dec_g(g[I.value] & 0xFFFFu);
            fb[I.value] = C::dec_g(g[I.value] >> 16);
        });
        collide_pair<V, COLL, float, SL, (FMT >= 2)>(a.k, f, fb);
        static_for<0, V::Q>([&](auto I) { g[I.value] = C::enc_g(f[I.value]) | (C::enc_g(fb[I.value]) << 16); });
    } else {
        static_for<0, V::Q>([&](auto I) { f[I.value] = C::dec_g(g[I.value] & 0xFFFFu); });
        collide<V, COLL, float, SL, (FMT >= 2)>(a.k, f);
        static_for<0, V::Q>([&](auto I) { g[I.value] = (g[I.value] & 0xFFFF0000u) | C::enc_g(f[I.value]); });
        static_for<0, V::Q>([&](auto I) { f[I.value] = C::dec_g(g[I.value] >> 16); });
        collide<V, COLL, float, SL, (FMT >= 2)>(a.k, f);
        static_for<0, V::Q>([&](auto I) { g[I.value] = (g[I.value] & 0xFFFFu) | (C::enc_g(f[I.value]) << 16); });
    }
    if (active) {
        uint16_t* dst = (uint16_t*)a.dst;
        const uint32_t n0 = (uint32_t)x0 + yo[1] + zo[1];
        static_for<0, V::Q>([&](auto I) {
            *reinterpret_cast<uint32_t*>(dst + (uint32_t)I.value * N + n0) = g[I.value];
        });
    }
}

// Pairs of codes: FP16 and FP16S convert two values per instruction.
template <int FMT> struct PairCodec {
    __device__ static float2 dec(uint32_t g) {
        return make_float2(Codec16<FMT>::dec_g(g & 0xFFFFu), Codec16<FMT>::dec_g(g >> 16));
    }
    __device__ static uint32_t enc(float lo, float hi) {
        return Codec16<FMT>::enc_g(lo) | (Codec16<FMT>::enc_g(hi) << 16);
    }
};
template <int FMT> struct PairCodecHalf {
    __device__ static float2 dec(uint32_t g) {
        __half2 h;
        memcpy(&h, &g, 4);
        return __half22float2(h);
    }
    __device__ static uint32_t enc(float lo, float hi) {   // round to nearest even, as __float2half_rn
        const __half2 h = __floats2half2_rn(lo, hi);
        uint32_t g;
        memcpy(&g, &h, 4);
        return g;
    }
};
template <> struct PairCodec<2> : PairCodecHalf<2> {};
template <> struct PairCodec<3> : PairCodecHalf<3> {};

// One step on the chunked layout, 16-bit storage, FP32 arithmetic: a warp
// owns one 64-cell chunk of a row (lane l: cells 2l and 2l+1) and moves every
// population as one 128-byte line of 32-bit code pairs, at a compile-time
// offset from the chunk of the source (or destination) row.  Needs nx a
// multiple of 64; block = 32 x by threads.  Per-cell arithmetic is
// cell_step's.
//   PHASE LAYOUT_AB: pull from copy A, write own cells in copy B.  Pairs
//     shifted in x are assembled by warp shuffles; lanes 0 and 31 read the
//     missing code from the neighbouring chunk (periodic in x).
//   PHASE LAYOUT_AA_SWAPPED (odd A-A half): pull slot opposite(i) of the
//     upstream cell the same way, push slot i of the downstream cell: a pair
//     shifted in x is assembled from this lane's and the neighbouring lane's
//     codes; the half that belongs to the neighbouring chunk is one 16-bit
//     store (every location is written by the warp whose cell read it).
//   PHASE LAYOUT_AA_NATURAL (even A-A half): read own slot i, write own slot
//     opposite(i); no shifts.
// PLAIN (flagged lattice): only cells whose flag byte is 0 are written, and
// in the A-B and even A-A halves the plain bounce-back cells (byte
// F_NEAR_SOLID); a pair with one such cell is written as a single 16-bit
// code; the other cells belong to the list kernel.
template <class V, int COLL, int FMT, int PHASE, bool PLAIN>
__global__ void __launch_bounds__(256, V::Q > 19 ? 2 : 3) k_step_pair_chunked(const StepArgs<float> a) {
    using PC = PairCodec<FMT>;
    constexpr int SL = Codec16<FMT>::SL;
    constexpr uint32_t CHE = (uint32_t)V::Q * CHUNK;     // codes per chunk
    // posits: the encoding table of the block (4 KB), filled before any warp leaves
    constexpr bool TAB = FMT >= 5 && FMT <= 9;
    __shared__ EncEntry tab[TAB ? 512 : 1];
    if constexpr (TAB) {
        const int t = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
        for (int i = t; i < 512; i += nt) tab[i] = kEncTable<FMT>.e[i];
        __syncthreads();
    }
    const int lane = threadIdx.x;
    const uint32_t X = blockIdx.x, XT = (uint32_t)a.nx / CHUNK;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (y >= a.ny) return;                                 // whole warps leave together
    const uint32_t ny = (uint32_t)a.ny;
    const uint32_t ry[3] = {(uint32_t)(y == 0 ? a.ny - 1 : y - 1), (uint32_t)y, (uint32_t)(y == a.ny - 1 ? 0 : y + 1)};
    const uint32_t rz[3] = {(uint32_t)(z == 0 ? a.nz - 1 : z - 1) * ny, (uint32_t)z * ny,
                            (uint32_t)(z == a.nz - 1 ? 0 : z + 1) * ny};
    // chunk offsets of the x-neighbouring chunks (periodic)
    const int32_t prev = X == 0 ? (int32_t)((XT - 1) * CHE) : -(int32_t)CHE;
    const int32_t next = X == XT - 1 ? -(int32_t)((XT - 1) * CHE) : (int32_t)CHE;
    const uint16_t* src = (const uint16_t*)a.src;
    uint16_t* dst = (uint16_t*)a.dst;
    const uint32_t own_chunk = (ry[1] + rz[1]) * XT + X;   // < 2^25: N < 2^31 cells
    // Blocks start in launch order (x, then y, then z), so the warp at the
    // same chunk a.pf planes and a.pf_y rows further runs about one wave
    // later: this warp sends that row's q lines (and, flagged, its flag
    // line) into L2 ahead of it.  Nothing waits on these prefetches, so they
    // keep HBM busy beyond the loads the registers of the resident warps can
    // hold; the bytes read from HBM stay the same.  Only the formats with
    // hardware conversion are bound by HBM; the others are bound by
    // instruction issue and skip it.
    if constexpr (FMT == 2 || FMT == 3) {
        int yf = y + a.pf_y, zf = z + a.pf;
        if (yf >= a.ny) { yf -= a.ny; ++zf; }
        if ((a.pf > 0 || a.pf_y > 0) && zf < a.nz) {
            const uint32_t fut = ((uint32_t)yf + (uint32_t)zf * ny) * XT + X;
            if (lane < V::Q) asm volatile("prefetch.global.L2 [%0];" ::"l"(src + (size_t)fut * CHE + lane * CHUNK));
            else if (PLAIN && lane == V::Q) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.flags + (size_t)fut * CHUNK));
        }
    }
    uint32_t pl = 3u;   // bit 0: cell 2l is updated here, bit 1: cell 2l + 1
    uint32_t bb = 0u;   // the same bits for plain bounce-back cells (A-B)
    if constexpr (PLAIN) {
        const uint32_t fl2 = reinterpret_cast<const uint16_t*>(a.flags)[own_chunk * (CHUNK / 2) + lane];
        const uint32_t f0 = fl2 & 0xFFu, f1 = fl2 >> 8;
        pl = (f0 == 0u ? 1u : 0u) | (f1 == 0u ? 2u : 0u);
        // plain bounce-back cells: A-B replaces their wall directions below;
        // the even A-A half treats them as plain; the odd half leaves them
        // to the list kernel (their pushes into solid cells turn back; doing
        // that here, with the turned-back pushes masked per direction, made
        // the in-place cavities 6% slower)
        if constexpr (PHASE != LAYOUT_AA_SWAPPED) {
            bb = (f0 == F_NEAR_SOLID ? 1u : 0u) | (f1 == F_NEAR_SOLID ? 2u : 0u);
            pl |= bb;
        }
        if (!__any_sync(0xffffffffu, pl != 0u)) return;   // nothing to update in this chunk
    }
    // Plain bounce-back (flagged A-B): a direction whose upstream cell is
    // solid takes the code of the cell's own opposite population.  A warp
    // with such cells copies its own row's code pairs into shared memory by
    // cp.async, and their lanes load their two wall masks, before the pulls
    // are issued; both are used after the pulls.  The copies hold no
    // registers meanwhile, so the pulls stay in flight together as in a warp
    // without such cells.
    constexpr bool BBS = PLAIN && PHASE == LAYOUT_AB;
    // [warp of the block][slot][lane]; the kernel is launched with 32 x 8 threads
    __shared__ uint32_t bbrow[BBS ? 8 : 1][BBS ? V::Q : 1][32];
    uint2 wm = make_uint2(0u, 0u);
    bool anybb = false;
    if constexpr (BBS) {
        anybb = __any_sync(0xffffffffu, bb != 0u);
        if (anybb) {   // every lane of the warp stages (a branch per lane measured slower than the copies it saves)
            if (bb != 0u) {
                const uint32_t n0 = (ry[1] + rz[1]) * (uint32_t)a.nx + X * CHUNK + 2u * (uint32_t)lane;   // cell 2l (even)
                wm = *reinterpret_cast<const uint2*>(a.walls + n0);
                if (!(bb & 1u)) wm.x = 0u;
                if (!(bb & 2u)) wm.y = 0u;
            }
            const uint32_t* ownw = reinterpret_cast<const uint32_t*>(src + (size_t)own_chunk * CHE) + lane;
            static_for<1, V::Q>([&](auto I) {
                const uint32_t sa = (uint32_t)__cvta_generic_to_shared(&bbrow[threadIdx.y][I.value][lane]);
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(ownw + I.value * (CHUNK / 2))
                             : "memory");
            });
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
    }
    uint32_t g[V::Q];   // lo half: cell 2*lane, hi half: cell 2*lane + 1 (of this chunk)
    if constexpr (PHASE == LAYOUT_AA_NATURAL) {
        const uint32_t* pairs = reinterpret_cast<const uint32_t*>(src + (size_t)own_chunk * CHE) + lane;
        static_for<0, V::Q>([&](auto I) { g[I.value] = pairs[I.value * (CHUNK / 2)]; });
    } else {
        // lane 0 reads code 63 of the previous chunk, lane 31 code 0 of the next one
        const int32_t adj = lane == 0 ? prev + (CHUNK - 1) : next;
        // loads grouped by source row (c_y, c_z): one pointer per row, the slot
        // offsets are compile-time
        static_for<0, 9>([&](auto RC) {
            constexpr int cyr = RC.value % 3 - 1, czr = RC.value / 3 - 1;
            const uint16_t* rowp = src + (size_t)((ry[1 - cyr] + rz[1 - czr]) * XT + X) * CHE;
            const uint32_t* pairs = reinterpret_cast<const uint32_t*>(rowp) + lane;
            const uint16_t* edge = rowp + adj;
            static_for<0, V::Q>([&](auto I) {
                constexpr int i = I.value, cx = V::c(i, 0);
                constexpr int slot = PHASE == LAYOUT_AA_SWAPPED ? opposite(i) : i;
                if constexpr (V::c(i, 1) == cyr && V::c(i, 2) == czr) {
                    const uint32_t P = pairs[slot * (CHUNK / 2)];
                    if constexpr (cx == 0) {
                        g[i] = P;
                    } else if constexpr (cx > 0) {      // sources 2l-1, 2l
                        const uint32_t Pu = __shfl_up_sync(0xffffffffu, P, 1);
                        const uint32_t e = lane == 0 ? (uint32_t)edge[slot * CHUNK] : (Pu >> 16);
                        g[i] = (P << 16) | e;
                    } else {                            // sources 2l+1, 2l+2
                        const uint32_t Pd = __shfl_down_sync(0xffffffffu, P, 1);
                        const uint32_t e = lane == 31 ? (uint32_t)edge[slot * CHUNK] : (Pd & 0xFFFFu);
                        g[i] = (P >> 16) | (e << 16);
                    }
                }
            });
        });
    }
    if constexpr (BBS) {
        if (anybb) {
            asm volatile("cp.async.wait_all;" ::: "memory");   // this lane's copies (each lane reads its own words)
            static_for<1, V::Q>([&](auto I) {
                constexpr int i = I.value;
                const uint32_t w0 = (wm.x >> i) & 1u, w1 = (wm.y >> i) & 1u;
                if (w0 | w1) {
                    const uint32_t o = bbrow[threadIdx.y][opposite(i)][lane];   // slot opposite(i), both cells
                    const uint32_t keep = (w0 ? 0u : 0x0000FFFFu) | (w1 ? 0u : 0xFFFF0000u);
                    g[i] = (g[i] & keep) | (o & ~keep);
                }
            });
        }
    }
    // SEQ: one cell at a time, the first cell's codes going back into g
    // before the second is decoded, so that only one cell's values are live:
    // for 27 populations (the register budget of 27 code pairs) and for the
    // software codecs (FP16C, posits), whose conversions need registers of
    // their own.  The formats with hardware conversion decode and encode both
    // cells as pairs.
    constexpr bool SEQ = V::Q > 19 || !(FMT == 2 || FMT == 3);
    auto enc1 = [&](float v) -> uint32_t {
        if constexpr (TAB) return enc_table(tab, v);
        else return Codec16<FMT>::enc_g(v);
    };
    float fa[V::Q], fb[SEQ ? 1 : V::Q];
    static_for<0, V::Q>([&](auto I) {
        if constexpr (SEQ) fa[I.value] = Codec16<FMT>::dec_g(g[I.value] & 0xFFFFu);
        else fa[I.value] = PC::dec(g[I.value]).x;
    });
    if constexpr (SEQ) {
        collide<V, COLL, float, SL, (FMT >= 2)>(a.k, fa);
        static_for<0, V::Q>([&](auto I) {
            g[I.value] = (g[I.value] & 0xFFFF0000u) | enc1(fa[I.value]);
            fa[I.value] = Codec16<FMT>::dec_g(g[I.value] >> 16);
        });
        collide<V, COLL, float, SL, (FMT >= 2)>(a.k, fa);
        static_for<0, V::Q>([&](auto I) { g[I.value] = (g[I.value] & 0xFFFFu) | (enc1(fa[I.value]) << 16); });
    } else {
        static_for<0, V::Q>([&](auto I) { fb[I.value] = PC::dec(g[I.value]).y; });
        collide_pair<V, COLL, float, SL, (FMT >= 2)>(a.k, fa, fb);
    }
    // the new code pair of population i
    auto pair = [&](auto I) -> uint32_t {
        if constexpr (SEQ) return g[I.value];
        else return PC::enc(fa[I.value], fb[I.value]);
    };
    // writes the pair w of 16-bit codes at element e (of line start `line`),
    // only the halves whose cells may be written (ok bit 0: lo, bit 1: hi)
    auto put = [&](uint16_t* line, int e, uint32_t w, uint32_t ok) {
        if (ok == 3u) *reinterpret_cast<uint32_t*>(line + e) = w;
        else if (ok == 1u) line[e] = (uint16_t)w;
        else if (ok == 2u) line[e + 1] = (uint16_t)(w >> 16);
    };
    if constexpr (PHASE != LAYOUT_AA_SWAPPED) {
        uint16_t* out = dst + (size_t)own_chunk * CHE + 2 * lane;
        static_for<0, V::Q>([&](auto I) {
            constexpr int slot = PHASE == LAYOUT_AA_NATURAL ? opposite(I.value) : I.value;
            const uint32_t w = pair(I);
            if constexpr (PLAIN) put(out + slot * CHUNK, 0, w, pl);
            else *reinterpret_cast<uint32_t*>(out + slot * CHUNK) = w;
        });
    } else {
        // push slot i into the destination row (y + c_y, z + c_z): its chunk
        // lies dy[c_y] + dz[c_z] chunks from this cell's own (periodic; |dy +
        // dz| < N / 64 < 2^25), four offsets kept through the collision
        // instead of the row indices
        const uint32_t pl_up = __shfl_up_sync(0xffffffffu, pl, 1), pl_dn = __shfl_down_sync(0xffffffffu, pl, 1);
        const int32_t rowc = (int32_t)XT, planec = (int32_t)(ny * XT);
        const int32_t dy[3] = {y == 0 ? (a.ny - 1) * rowc : -rowc, 0, y == a.ny - 1 ? -(a.ny - 1) * rowc : rowc};
        const int32_t dz[3] = {z == 0 ? (a.nz - 1) * planec : -planec, 0, z == a.nz - 1 ? -(a.nz - 1) * planec : planec};
        uint16_t* const base = dst + (size_t)own_chunk * CHE;
        static_for<0, V::Q>([&](auto I) {
            constexpr int i = I.value, cx = V::c(i, 0), cy = V::c(i, 1), cz = V::c(i, 2);
            uint16_t* rowp = base + (int64_t)(dy[1 + cy] + dz[1 + cz]) * (int64_t)CHE + i * CHUNK;
            const uint32_t own = pair(I);
            if constexpr (cx == 0) {
                if constexpr (PLAIN) put(rowp, 2 * lane, own, pl);
                else *reinterpret_cast<uint32_t*>(rowp + 2 * lane) = own;
            } else if constexpr (cx > 0) {            // cells 2l-1, 2l land on 2l, 2l+1
                const uint32_t up = __shfl_up_sync(0xffffffffu, own, 1);
                const uint32_t w = __byte_perm(up, own, 0x5432);
                const uint32_t ok = (lane == 0 ? 0u : ((pl_up >> 1) & 1u)) | ((pl & 1u) << 1);
                put(rowp, 2 * lane, w, ok);
                if (lane == 31 && (pl & 2u)) rowp[next + 0] = (uint16_t)(own >> 16);   // cell 63 -> next chunk
            } else {                                  // cells 2l+1, 2l+2 land on 2l, 2l+1
                const uint32_t dn = __shfl_down_sync(0xffffffffu, own, 1);
                const uint32_t w = __byte_perm(own, dn, 0x5432);
                const uint32_t ok = ((pl >> 1) & 1u) | (lane == 31 ? 0u : ((pl_dn & 1u) << 1));
                put(rowp, 2 * lane, w, ok);
                if (lane == 0 && (pl & 1u)) rowp[prev + (CHUNK - 1)] = (uint16_t)own;   // cell 0 -> previous chunk
            }
        });
    }
}

// ---------------------------------------------------------------- ensemble
// Many independent lattices in one launch.  Each member's cells, in linear
// order n = x + nx (y + ny z), are cut into tiles of blockDim.x consecutive
// cells; tile_member[b] names the member of block b.  Coordinates come from n
// by multiply-high division with per-member magic numbers (exact for n < 2^31).
struct FastDiv {
    uint32_t magic, shift, one;   // one != 0: divisor 1
    __device__ __forceinline__ uint32_t div(uint32_t n) const {
        return one ? n : (__umulhi(n, magic) >> shift);
    }
};

template <class R> struct EnsMember {
    StepArgs<R> args[2];       // args[p]: arguments for a step of parity p
    uint32_t ncells, tile0;    // cells, first global tile of this member
    FastDiv by_plane, by_nx;
    uint32_t open;             // a face of the lattice holds non-solid cells (periodic or open faces)
};

// L2 prefetch for the tile a.pf tiles further in launch order (about one
// wave later, since blocks start in launch order): its population codes and
// its flag bytes, one 128-byte line per thread; the bytes read from HBM stay
// the same.  Structure of arrays: q ranges of the tile's cells; chunked
// (CH): the whole chunks that hold its cells, q lines each.  16-bit formats
// with hardware conversion only (HBM-bound).
template <class V, int FMT, bool CH, class R>
__device__ __forceinline__ void prefetch_tile_ahead(const EnsMember<R>* __restrict__ members,
                                                    const uint32_t* __restrict__ tile_member, int parity, int pf) {
    if constexpr (FMT == 2 || FMT == 3) {
        using T = typename Storage<FMT>::T;
        constexpr uint32_t LINE = 128 / sizeof(T);
        const uint32_t ft = blockIdx.x + (uint32_t)pf;
        if (pf <= 0 || ft >= gridDim.x) return;
        const uint32_t t = threadIdx.x;
        // threads beyond the most lines a tile can need leave before the
        // member lookup (a tile of blockDim cells spans at most
        // blockDim / 64 + 2 chunks; a population range at most `per` lines)
        const uint32_t per = (blockDim.x + LINE - 1) / LINE + 1;
        if (t >= (CH ? (blockDim.x / CHUNK + 2u) * (uint32_t)V::Q : (uint32_t)V::Q * per) + 2u) return;
        const EnsMember<R>& F = members[__ldg(tile_member + ft)];
        const uint32_t n0 = (ft - F.tile0) * blockDim.x;
        const uint32_t last = min(blockDim.x, F.ncells - n0) - 1;   // tile ft holds cells n0 .. n0 + last
        const T* src = (const T*)F.args[parity].src;
        uint32_t lines;                                              // population lines of the tile
        if constexpr (CH) {
            static_assert(CHUNK == LINE, "a chunk slot is one line");
            const uint32_t c0 = n0 / CHUNK, c1 = (n0 + last) / CHUNK;
            lines = (c1 - c0 + 1u) * (uint32_t)V::Q;
            if (t < lines) asm volatile("prefetch.global.L2 [%0];" ::"l"(src + ((size_t)c0 * V::Q * CHUNK + (size_t)t * LINE)));
        } else {
            // `per` lines per population range: one more than whole lines, for
            // a range that does not start on a line boundary
            lines = V::Q * per;
            if (t < lines) {
                const uint32_t i = t / per, k = t - i * per;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(src + (size_t)i * F.ncells + n0 + min(k * LINE, last)));
            }
        }
        if (t >= lines && t < lines + 2u && F.args[parity].flags)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(F.args[parity].flags + n0 + min((t - lines) * 128u, last)));
    }
}

// The plain cells (flag byte 0) of every member; the others come from the
// ensemble's list (k_ensemble_list).  CH: members on the chunked layout.
template <class V, int COLL, int FMT, class R, int SCHEME, class IX, bool CH = false>
__global__ void __launch_bounds__(256, sizeof(R) == 8 ? 2 : (COLL == 2 ? 3 : 4)) k_ensemble_step(const EnsMember<R>* __restrict__ members,
                                                        const uint32_t* __restrict__ tile_member, int parity) {
    const EnsMember<R>& M = members[__ldg(tile_member + blockIdx.x)];
    prefetch_tile_ahead<V, FMT, CH>(members, tile_member, parity, M.args[parity].pf);
    const uint32_t n = (blockIdx.x - M.tile0) * blockDim.x + threadIdx.x;
    if (n >= M.ncells) return;
    const StepArgs<R> a = M.args[parity];
    const uint32_t z = M.by_plane.div(n);
    const uint32_t r = n - z * (uint32_t)(a.nx * a.ny);
    const uint32_t y = M.by_nx.div(r);
    const uint32_t x = r - y * (uint32_t)a.nx;
    cell_step<V, COLL, FMT, R, SCHEME, false, IX, true, CH>(a, (int)x, (int)y, (int)z);
}

// Paired ensemble step, A-B, 16-bit storage with hardware conversion (FP16,
// FP16S), FP32 arithmetic, members on the structure-of-arrays layout: one warp
// per run of 64 consecutive cells of a member (lane l: cells 2l, 2l + 1 of
// the run), every population moved as 32-bit pairs of codes.  Population i of
// cell n streams from the cell n - d_i, d_i = c_ix + nx (c_iy + ny c_iz), which
// is its upstream neighbour for every cell off the lattice's faces.  A source
// pair that starts at an odd element is this lane's upper code and the next
// lane's lower one (lane 31 reads the missing code); a destination pair at an
// odd element (i N odd) is written as the word of the previous lane's upper
// and this lane's lower code, with the codes that cross into the neighbouring
// runs as single 16-bit stores.  Updated here: plain cells (flag byte 0) and
// plain bounce-back cells (F_NEAR_SOLID) off the faces; in a member with
// non-solid face cells those take the per-cell path; the listed cells follow
// in k_ensemble_list.  Lanes without a cell to update read in-range elements
// (clamped) and write nothing.
// the per-cell update of a cell on a lattice face (wrapped neighbours), kept
// out of line so that the paired kernel's registers serve its common path
template <class V, int COLL, int FMT, bool CH>
__device__ __noinline__ void ensemble_face_cell(const StepArgs<float>& a, int x, int y, int z) {
    cell_step<V, COLL, FMT, float, SCHEME_AB, false, uint32_t, true, CH>(a, x, y, z);
}

// element of slot i of cell m: structure of arrays (i N + m), or chunked
// (chunk m / 64 holds its q slots of 64 codes: ((m/64) q + i) 64 + m % 64)
template <class V, bool CH>
__device__ __forceinline__ uint32_t ens_elem(int i, uint32_t m, uint32_t N) {
    if constexpr (CH) return m + (m >> 6) * (uint32_t)((V::Q - 1) * CHUNK) + (uint32_t)(i * CHUNK);
    else return (uint32_t)i * N + m;
}

template <class V, int COLL, int FMT, bool CH>
__global__ void __launch_bounds__(128, 5) k_ensemble_pair(const EnsMember<float>* __restrict__ members,
                                                          const uint32_t* __restrict__ tile_member, int parity) {
    using PC = PairCodec<FMT>;
    constexpr int SL = Codec16<FMT>::SL;
    const EnsMember<float>& M = members[__ldg(tile_member + blockIdx.x)];
    const int lane = threadIdx.x;
    const uint32_t run = (blockIdx.x - M.tile0) * blockDim.y + threadIdx.y;
    const uint32_t N = M.ncells;
    if (run * 64u >= N) return;                                   // whole warps leave
    const StepArgs<float>& a = M.args[parity];                    // read in place (uniform loads)
    // L2 prefetch of the run a.pf tiles further in launch order (about one
    // wave later): its q population ranges and its flags, one line per lane
    if constexpr (FMT == 2 || FMT == 3) {
        const uint32_t ft = blockIdx.x + (uint32_t)a.pf;
        if (a.pf > 0 && ft < gridDim.x) {
            const EnsMember<float>& F = members[__ldg(tile_member + ft)];
            const uint32_t fr = (ft - F.tile0) * blockDim.y + threadIdx.y;
            if (fr * 64u < F.ncells) {
                const uint16_t* fs = (const uint16_t*)F.args[parity].src;
                if (lane < V::Q) asm volatile("prefetch.global.L2 [%0];" ::"l"(fs + ens_elem<V, CH>(lane, fr * 64u, F.ncells)));
                else if (lane == V::Q) asm volatile("prefetch.global.L2 [%0];" ::"l"(F.args[parity].flags + fr * 64u));
            }
        }
    }
    const uint32_t n = run * 64u + 2u * (uint32_t)lane;          // the lane's first cell
    const uint32_t f0 = n < N ? (uint32_t)a.flags[n] : F_WALL;
    const uint32_t f1 = n + 1u < N ? (uint32_t)a.flags[n + 1u] : F_WALL;
    uint32_t pl = (f0 == 0u ? 1u : 0u) | (f1 == 0u ? 2u : 0u);             // updated here: plain ...
    uint32_t bb = (f0 == F_NEAR_SOLID ? 1u : 0u) | (f1 == F_NEAR_SOLID ? 2u : 0u);   // ... and bounce-back
    // halves the stores leave alone: solid cells and cells past the member
    // (their populations stay zero) and cells the per-cell path updated
    uint32_t skip = ((f0 & F_WALL) ? 1u : 0u) | ((f1 & F_WALL) ? 2u : 0u);
    const uint32_t plane = (uint32_t)a.nx * (uint32_t)a.ny;
    if (M.open && ((pl | bb) != 0u)) {
        // cells on a face need wrapped neighbours: the per-cell path
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            if (!(((pl | bb) >> h) & 1u)) continue;
            const uint32_t c = n + (uint32_t)h;
            const uint32_t z = M.by_plane.div(c), r = c - z * plane, y = M.by_nx.div(r), x = r - y * (uint32_t)a.nx;
            if (x == 0u || x + 1u == (uint32_t)a.nx || y == 0u || y + 1u == (uint32_t)a.ny || z == 0u ||
                z + 1u == (uint32_t)a.nz) {
                ensemble_face_cell<V, COLL, FMT, CH>(a, (int)x, (int)y, (int)z);
                pl &= ~(1u << h);
                bb &= ~(1u << h);
                skip |= 1u << h;
            }
        }
    }
    if (!__any_sync(0xffffffffu, (pl | bb) != 0u)) return;
    const uint16_t* src = (const uint16_t*)a.src;
    uint16_t* dst = (uint16_t*)a.dst;
    // start of the copy's last whole aligned word (chunked: padded to whole
    // chunks; structure of arrays: q N may be odd, the last code then has no
    // aligned partner and the clamp stops one word earlier)
    const uint32_t qN2 = ((uint32_t)V::Q * (CH ? ((N + 63u) & ~63u) : N) - 2u) & ~1u;
    uint32_t g[V::Q];
    static_for<0, V::Q>([&](auto I) {
        constexpr int i = I.value, cx = V::c(i, 0), cy = V::c(i, 1), cz = V::c(i, 2);
        const int32_t d = cx + cy * a.nx + cz * (int32_t)plane;
        const uint32_t m = n - (uint32_t)d;                       // the first cell's source cell
        // the aligned word holding element e of the source; lanes whose cells
        // are not updated here may compute an element outside the copy, which
        // the clamp brings back in (their codes are not used)
        const uint32_t e = ens_elem<V, CH>(i, m, N);
        const uint32_t es = min(e & ~1u, qN2);
        const uint32_t w = *reinterpret_cast<const uint32_t*>(src + es);
        // the parity of e is the same in every lane (warp-uniform branch)
        const bool odd = CH ? ((uint32_t)d & 1u) : ((((uint32_t)i * N - (uint32_t)d) & 1u) != 0u);
        if (!odd) {
            g[i] = w;
        } else {                                                    // codes e, e + 1: hi of w, lo of the next word
            uint32_t nxt = __shfl_down_sync(0xffffffffu, w, 1);
            if (lane == 31) nxt = (uint32_t)src[min(ens_elem<V, CH>(i, m + 1u, N), qN2 + 1u)];
            g[i] = __byte_perm(w, nxt, 0x5432);
        }
    });
    // plain bounce-back: a direction whose upstream cell is solid takes the
    // code of the cell's own opposite population
    if (__any_sync(0xffffffffu, bb != 0u)) {
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            if (!((bb >> h) & 1u)) continue;
            const uint32_t c = n + (uint32_t)h;
            const uint32_t walls = a.walls[c];
            static_for<1, V::Q>([&](auto I) {
                constexpr int i = I.value;
                if ((walls >> i) & 1u) {
                    const uint32_t cc = src[ens_elem<V, CH>(opposite(i), c, N)];
                    g[i] = h ? ((g[i] & 0xFFFFu) | (cc << 16)) : ((g[i] & 0xFFFF0000u) | cc);
                }
            });
        }
    }
    float fa[V::Q], fb[V::Q];
    static_for<0, V::Q>([&](auto I) {
        const float2 v = PC::dec(g[I.value]);
        fa[I.value] = v.x;
        fb[I.value] = v.y;
    });
    const Relax<float> k = a.k;                                   // the member's constants in registers
    collide_pair<V, COLL, float, SL, (FMT >= 2)>(k, fa, fb);
    // Every other half is written: the listed cells' halves carry values the
    // list launch that follows overwrites, so the stores are whole words,
    // the skipped halves masked to zero, except where a word would reach
    // past the member (structure of arrays) or into a skipped cell the per-cell
    // path wrote.
    const uint32_t keep = ((skip & 1u) ? 0u : 0x0000FFFFu) | ((skip & 2u) ? 0u : 0xFFFF0000u);
    const bool face_done = M.open != 0u && skip != (((f0 & F_WALL) ? 1u : 0u) | ((f1 & F_WALL) ? 2u : 0u));
    const uint32_t w3 = (skip == 3u) ? 0u : (face_done || (!CH && n + 1u >= N) ? (skip ^ 3u) : 3u);
    const uint32_t w3_up = __shfl_up_sync(0xffffffffu, w3, 1);
    static_for<0, V::Q>([&](auto I) {
        constexpr int i = I.value;
        const uint32_t own = PC::enc(fa[i], fb[i]) & keep;
        const uint32_t e = ens_elem<V, CH>(i, n, N);
        if (CH || (((uint32_t)i * N) & 1u) == 0u) {                // warp-uniform: aligned pair
            if (w3 == 3u) *reinterpret_cast<uint32_t*>(dst + e) = own;
            else if (w3 == 1u) dst[e] = (uint16_t)own;
            else if (w3 == 2u) dst[e + 1u] = (uint16_t)(own >> 16);
        } else {                                                    // word e-1: previous lane's upper, own lower code
            const uint32_t up = __shfl_up_sync(0xffffffffu, own, 1);
            const uint32_t okw = (lane == 0 ? 0u : ((w3_up >> 1) & 1u)) | ((w3 & 1u) << 1);
            const uint32_t w = __byte_perm(up, own, 0x5432);
            if (okw == 3u) *reinterpret_cast<uint32_t*>(dst + e - 1u) = w;
            else if (okw == 2u) dst[e] = (uint16_t)own;
            else if (okw == 1u) dst[e - 1u] = (uint16_t)(up >> 16);
            if (lane == 31 && (w3 & 2u)) dst[e + 1u] = (uint16_t)(own >> 16);   // cell n + 1: the next run's word
        }
    });
}

// The non-plain cells of all members: entry = member << 32 | cell.
template <class V, int COLL, int FMT, class R, int SCHEME, class IX, bool CH = false>
__global__ void __launch_bounds__(256) k_ensemble_list(const EnsMember<R>* __restrict__ members,
                                                        const uint64_t* __restrict__ cells, uint32_t count,
                                                        int parity) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const uint64_t e = cells[t];
    const EnsMember<R>& M = members[(uint32_t)(e >> 32)];
    const uint32_t n = (uint32_t)e;
    const StepArgs<R> a = M.args[parity];
    const uint32_t z = M.by_plane.div(n);
    const uint32_t r = n - z * (uint32_t)(a.nx * a.ny);
    const uint32_t y = M.by_nx.div(r);
    const uint32_t x = r - y * (uint32_t)a.nx;
    cell_step<V, COLL, FMT, R, SCHEME, true, IX, false, CH, false>(a, (int)x, (int)y, (int)z);
}

// ---------------------------------------------------------------- probes
// Per-cell quantities from the streamed populations: fields (rho, u with the
// Guo half-force), the populations themselves, or FP64 mass / energy sums.
// The cells are the planes z0..z1-1, or the listed cell indices when `cells`
// is set (every index already checked to lie in [0, N) by the host).
template <class R> struct ProbeArgs {
    StepArgs<R> a;
    int z0, z1;               // z-range handled by this launch
    double* out;              // FIELDS: 4 x count doubles; F: q x count doubles
    double* partial;          // REDUCE: 2 doubles per block
    const int64_t* cells;     // optional list of cell indices
    uint32_t ncells;          // its length
};

template <class V, int FMT, class R, int LAYOUT>
__global__ void __launch_bounds__(256) k_probe(const ProbeArgs<R> p, int mode) {
    const StepArgs<R>& a = p.a;
    const uint32_t plane = (uint32_t)a.nx * (uint32_t)a.ny;
    const uint32_t count = p.cells ? p.ncells : plane * (uint32_t)(p.z1 - p.z0);
    double m_acc = 0.0, e_acc = 0.0;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
        const uint32_t n = p.cells ? (uint32_t)p.cells[t] : (uint32_t)p.z0 * plane + t;
        const int z = (int)(n / plane);
        const uint32_t r = n - (uint32_t)z * plane;
        const int y = (int)(r / (uint32_t)a.nx);
        const int x = (int)(r - (uint32_t)y * a.nx);
        const uint32_t fl = a.flags ? a.flags[n] : 0u;
        const bool solid = fl & F_WALL;
        R f[V::Q];
        if (!solid) {
            if (a.flags) gather<V, FMT, R, true, LAYOUT>(a, (const typename Storage<FMT>::T*)a.src, x, y, z, n, fl, f);
            else gather<V, FMT, R, false, LAYOUT>(a, (const typename Storage<FMT>::T*)a.src, x, y, z, n, fl, f);
        }
        constexpr int SL = Storage<FMT>::SL;
        if (mode == PROBE_F) {
            static_for<0, V::Q>([&](auto I) {
                const R v = SL == 0 ? f[I.value] : f[I.value] * R(Pow2<SL>::down);
                p.out[(size_t)I.value * count + t] = solid ? 0.0 : (double)v;
            });
            continue;
        }
        double rho = 1.0, u[3] = {0.0, 0.0, 0.0};
        if (solid) {
        } else if (fl & F_EQ) {
            rho = (double)a.node_rho[n];
            for (int d = 0; d < 3; ++d) u[d] = (double)a.node_u[(size_t)d * a.N + n];
        } else {
            R rr, j[3], uu[3];
            moments<V, R, SL>(f, rr, j, a.k.sh);
            velocity<R, SL>(a.k, rr, j, uu);
            rho = (double)rr;
            for (int d = 0; d < 3; ++d) u[d] = (double)uu[d];
        }
        if (mode == PROBE_FIELDS) {
            p.out[t] = rho;
            p.out[(size_t)count + t] = u[0];
            p.out[2 * (size_t)count + t] = u[1];
            p.out[3 * (size_t)count + t] = u[2];
        } else if (!solid) {
            m_acc += rho;
            e_acc += 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        }
    }
    if (mode != PROBE_REDUCE) return;
    // block reduction in FP64 (fixed order: deterministic)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m_acc += __shfl_down_sync(0xffffffffu, m_acc, o);
        e_acc += __shfl_down_sync(0xffffffffu, e_acc, o);
    }
    __shared__ double sm[2][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sm[0][warp] = m_acc; sm[1][warp] = e_acc; }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        m_acc = lane < nw ? sm[0][lane] : 0.0;
        e_acc = lane < nw ? sm[1][lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            m_acc += __shfl_down_sync(0xffffffffu, m_acc, o);
            e_acc += __shfl_down_sync(0xffffffffu, e_acc, o);
        }
        if (lane == 0) {
            p.partial[2 * blockIdx.x] = m_acc;
            p.partial[2 * blockIdx.x + 1] = e_acc;
        }
    }
}

// ---------------------------------------------------------------- put
// Initial populations for cells of planes z0..z1-1 from device doubles:
// INIT: shifted equilibrium (Sec. 2.2) of (rho, ux, uy, uz), each `count`
// doubles or NULL (rho = 1, u = 0); SETF: post-collision populations in[0]
// (q x count doubles).  Solid cells get zero.  A-A stores in the swapped
// layout (slot opposite(i)).
template <class R> struct PutArgs {
    StepArgs<R> a;
    int z0, z1;
    const double* in[4];
};

// PUT_LAYOUT bit 0: A-A (swapped slots), bit 1: chunked
template <class V, int FMT, class R, int PUT_LAYOUT>
__global__ void __launch_bounds__(256) k_put(const PutArgs<R> p, int setf) {
    constexpr bool AA = (PUT_LAYOUT & 1) != 0;
    constexpr bool CH = (PUT_LAYOUT & 2) != 0;
    using S = Storage<FMT>;
    const StepArgs<R>& a = p.a;
    const uint32_t plane = (uint32_t)a.nx * (uint32_t)a.ny;
    const uint32_t count = plane * (uint32_t)(p.z1 - p.z0);
    typename S::T* dst = (typename S::T*)a.dst;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
        const uint32_t n = (uint32_t)p.z0 * plane + t;
        const bool solid = a.flags && (a.flags[n] & F_WALL);
        R f[V::Q];
        if (setf) {
            static_for<0, V::Q>([&](auto I) { f[I.value] = (R)p.in[0][(size_t)I.value * count + t]; });
        } else {
            const R rho = p.in[0] ? (R)p.in[0][t] : R(1);
            const R u[3] = {p.in[1] ? (R)p.in[1][t] : R(0), p.in[2] ? (R)p.in[2][t] : R(0),
                            (V::D == 3 && p.in[3]) ? (R)p.in[3][t] : R(0)};
            equilibrium_only<V, R, 0>(rho, u, f, a.k.sh);
        }
        static_for<0, V::Q>([&](auto I) {
            constexpr int slot = AA ? opposite(I.value) : I.value;
            const size_t e = CH ? (size_t)chunk_elem<V>(slot, n) : (size_t)slot * a.N + n;
            S::template store<R>(dst, e, solid ? R(0) : f[I.value]);
        });
    }
}

// Sets the internal bits of non-solid cells: F_NEAR_SOLID if any neighbour
// is solid or the cell is an outflow cell, F_NEAR_MOVING if any neighbour is a
// moving wall.
// The wall mask of each cell (bit i: the upstream cell n - c_i is solid; 0
// for solid cells) goes to walls[n], so that the fast kernels replace the
// bounce-back directions of a cell from one word instead of q - 1 flag loads.
template <class V>
__global__ void k_mark_neighbours(uint8_t* flags, uint32_t* walls, int nx, int ny, int nz) {
    const uint32_t plane = (uint32_t)nx * (uint32_t)ny;
    const uint32_t N = plane * (uint32_t)nz;
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const uint32_t fl = flags[n];
        if (fl & F_WALL) {
            walls[n] = 0u;
            continue;
        }
        const int z = (int)(n / plane);
        const uint32_t r = n - (uint32_t)z * plane;
        const int y = (int)(r / (uint32_t)nx);
        const int x = (int)(r - (uint32_t)y * nx);
        const Nbr nb(x, y, z, nx, ny, nz);
        uint32_t any = 0, m = 0;
        static_for<1, V::Q>([&](auto I) {
            const uint32_t u = flags[nb.up<V, I.value>()];
            any |= u;
            m |= (u & F_WALL) ? (1u << I.value) : 0u;
        });
        walls[n] = m;
        // only the user bits of the neighbours are read (other threads add
        // internal bits to the bytes meanwhile)
        uint32_t add = 0;
        if ((any & F_WALL) || (fl & F_OUTFLOW)) add |= F_NEAR_SOLID;
        if (any & F_FREESLIP) add |= F_NEAR_FREESLIP;
        if (any & F_MOVING) add |= F_NEAR_MOVING;
        if (add) flags[n] = (uint8_t)(fl | add);
    }
}

}  // namespace lbm
