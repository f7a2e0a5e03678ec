// Ensembles: many independent lattices of uneven size advanced by ONE kernel
// launch per time step.  The members' cells are cut into tiles of `tile`
// consecutive cells (one thread block each); a per-tile table names the
// member, and a device table holds each member's pointers, sizes,
// relaxation constants and division magic numbers.  Steps are replayed from a CUDA graph of
// kGraphSteps launches.  Every cell runs the same per-cell routine as the
// single-lattice kernel, so results are bit-for-bit those of one launch per
// member.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "lbm.h"
#include "lbm_handle.h"

using namespace lbm;

namespace {
constexpr int kGraphSteps = 64;
}

// What the ensemble's tables took from a member: its copies, flags, node
// arrays and cell list, layout and scheme.  A member changed outside the
// ensemble (a new geometry, scheme or layout) no longer matches.
struct MemberKey {
    const void* f[2];
    const void* flags;
    const void* node_u;
    const void* node_rho;
    const void* special;
    uint32_t n_complex;
    int chunked, scheme;
    uint64_t geom_gen;
    explicit MemberKey(const lbm_handle* h = nullptr)
        : f{h ? h->f[0] : nullptr, h ? h->f[1] : nullptr}, flags(h ? h->flags : nullptr),
          node_u(h ? h->node_u : nullptr), node_rho(h ? h->node_rho : nullptr), special(h ? h->special : nullptr),
          n_complex(h ? h->n_complex : 0u), chunked(h ? h->chunked : 0), scheme(h ? h->p.scheme : 0),
          geom_gen(h ? h->geom_gen : 0u) {}
    bool operator==(const MemberKey& o) const {
        return f[0] == o.f[0] && f[1] == o.f[1] && flags == o.flags && node_u == o.node_u && node_rho == o.node_rho &&
               special == o.special && n_complex == o.n_complex && chunked == o.chunked && scheme == o.scheme &&
               geom_gen == o.geom_gen;
    }
};

struct lbm_ensemble {
    std::vector<lbm_handle*> m;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;
    KernelSet* ks = nullptr;
    bool fp64 = false, aa = false;
    void* table = nullptr;          // EnsMember<R>[count]
    uint64_t* list = nullptr;       // non-plain cells of all members: member << 32 | cell
    uint32_t n_list = 0;
    uint32_t* tile_member = nullptr;
    size_t table_bytes = 0, tiles_alloc = 0;
    int total_tiles = 0;
    int tile = 256;                 // cells per tile (per-cell kernel: = threads per block)
    int variant = LBM_ENS_PER_CELL; // LBM_ENS_PER_CELL or LBM_ENS_PAIRED
    int layout = LBM_LAYOUT_SOA;    // the members' layout: LBM_LAYOUT_SOA or LBM_LAYOUT_CHUNKED
    int warps = 4;                  // paired kernel: warps (runs of 64 cells) per tile
    std::vector<uint32_t> open;     // per member: a face holds non-solid cells
    bool idx32 = true;              // every member's q*N < 2^32
    int64_t s = 0;                  // steps taken through the ensemble
    std::vector<int64_t> t0;        // member step counters at creation
    std::vector<MemberKey> keys;    // the members as the tables hold them
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    std::vector<cudaStream_t> member_streams;   // the members' own streams other than `stream`
    cudaEvent_t order = nullptr;                // orders those streams against `stream`
    std::string err;

    lbm_status cuda(cudaError_t e, const char* what) {
        if (e == cudaSuccess) return LBM_OK;
        err = std::string(what) + ": " + cudaGetErrorString(e);
        return LBM_ERR_CUDA;
    }
    void drop_graphs() {
        for (auto& g : graph)
            if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    }
};

namespace {

// Members run their own calls (readbacks, layout and scheme changes) on their
// own streams and the ensemble's launches go to `stream`: to_ensemble makes
// `stream` wait for the work queued so far on the members' streams, the
// reverse makes the members' streams wait for the ensemble's work.  Nothing
// blocks the host.
lbm_status order_streams(lbm_ensemble* e, bool to_ensemble) {
    if (e->member_streams.empty()) return LBM_OK;
    if (!e->order && e->cuda(cudaEventCreateWithFlags(&e->order, cudaEventDisableTiming), "event")) return LBM_ERR_CUDA;
    if (to_ensemble) {
        for (cudaStream_t s : e->member_streams)
            if (e->cuda(cudaEventRecord(e->order, s), "event record") ||
                e->cuda(cudaStreamWaitEvent(e->stream, e->order, 0), "stream wait"))
                return LBM_ERR_CUDA;
        return LBM_OK;
    }
    if (e->cuda(cudaEventRecord(e->order, e->stream), "event record")) return LBM_ERR_CUDA;
    for (cudaStream_t s : e->member_streams)
        if (e->cuda(cudaStreamWaitEvent(s, e->order, 0), "stream wait")) return LBM_ERR_CUDA;
    return LBM_OK;
}

// sets *out if a cell on a face of the lattice is not solid
__global__ void k_face_open(const uint8_t* __restrict__ flags, int nx, int ny, int nz, int* out) {
    const uint32_t plane = (uint32_t)nx * (uint32_t)ny, N = plane * (uint32_t)nz;
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const uint32_t z = n / plane, r = n - z * plane, y = r / (uint32_t)nx, x = r - y * (uint32_t)nx;
        const bool face = x == 0 || x + 1 == (uint32_t)nx || y == 0 || y + 1 == (uint32_t)ny || z == 0 ||
                          z + 1 == (uint32_t)nz;
        if (face && !(flags[n] & lbm::F_WALL)) atomicOr(out, 1);
    }
}

__global__ void k_tag_cells(const uint32_t* __restrict__ cells, uint32_t count, uint32_t member, uint64_t* out) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x)
        out[t] = ((uint64_t)member << 32) | cells[t];
}

// floor(n / d) = umulhi(n, magic) >> shift for every n < 2^31 (d >= 2):
// shift + 32 = 31 + ceil(log2 d), magic = ceil(2^(31 + ceil(log2 d)) / d)
FastDiv make_div(uint32_t d) {
    FastDiv f{0u, 0u, 0u};
    if (d <= 1) { f.one = 1u; return f; }
    uint32_t lg = 0;
    while ((1ull << lg) < d) ++lg;
    const unsigned long long num = 1ull << (31 + lg);
    f.magic = (uint32_t)((num + d - 1) / d);
    f.shift = lg - 1;
    return f;
}

template <class R>
std::vector<EnsMember<R>> make_table(lbm_ensemble* e, std::vector<uint32_t>& tile_member) {
    std::vector<EnsMember<R>> tab(e->m.size());
    tile_member.clear();
    uint32_t total = 0;
    for (size_t k = 0; k < e->m.size(); ++k) {
        lbm_handle* h = e->m[k];
        const Relax<R>* rk_ptr;
        if constexpr (std::is_same<R, double>::value) rk_ptr = &h->kd; else rk_ptr = &h->kf;
        const Relax<R>& rk = *rk_ptr;
        EnsMember<R>& M = tab[k];
        M.args[0] = h->args(rk, e->aa ? 0 : h->cur);
        M.args[1] = h->args(rk, e->aa ? 0 : 1 - h->cur);
        // L2 prefetch distance in tiles: the tiles that fit on the GPU at once
        // (paired kernel: 20 warps per SM)
        M.args[0].pf = M.args[1].pf =
            e->variant == LBM_ENS_PAIRED ? h->num_sms * (20 / e->warps) : h->num_sms * (2048 / e->tile);
        M.ncells = (uint32_t)h->N;
        M.tile0 = total;
        M.by_plane = make_div((uint32_t)h->plane());
        M.by_nx = make_div((uint32_t)h->p.nx);
        M.open = e->open[k];
        const uint32_t tile_cells = e->variant == LBM_ENS_PAIRED ? 64u * (uint32_t)e->warps : (uint32_t)e->tile;
        const uint32_t tiles = (uint32_t)((h->N + tile_cells - 1) / tile_cells);
        tile_member.insert(tile_member.end(), tiles, (uint32_t)k);
        total += tiles;
    }
    e->total_tiles = (int)total;
    return tab;
}

lbm_status upload_table(lbm_ensemble* e) {
    std::vector<uint32_t> tiles;
    size_t bytes;
    const void* src;
    std::vector<EnsMember<float>> tf;
    std::vector<EnsMember<double>> td;
    if (e->fp64) { td = make_table<double>(e, tiles); src = td.data(); bytes = td.size() * sizeof(EnsMember<double>); }
    else { tf = make_table<float>(e, tiles); src = tf.data(); bytes = tf.size() * sizeof(EnsMember<float>); }
    if (order_streams(e, true) != LBM_OK) return LBM_ERR_CUDA;   // members' relayouts and scheme swaps first
    if (e->cuda(cudaStreamSynchronize(e->stream), "sync")) return LBM_ERR_CUDA;
    if (!e->table) {
        if (e->cuda(cudaMalloc(&e->table, bytes), "table alloc")) return LBM_ERR_OOM;
        e->table_bytes = bytes;
    }
    if (tiles.size() > e->tiles_alloc) {
        if (e->tile_member) cudaFree(e->tile_member);
        e->tile_member = nullptr;
        if (e->cuda(cudaMalloc((void**)&e->tile_member, tiles.size() * sizeof(uint32_t)), "table alloc"))
            return LBM_ERR_OOM;
        e->tiles_alloc = tiles.size();
    }
    if (e->cuda(cudaMemcpyAsync(e->table, src, bytes, cudaMemcpyHostToDevice, e->stream), "table upload"))
        return LBM_ERR_CUDA;
    if (e->cuda(cudaMemcpyAsync(e->tile_member, tiles.data(), tiles.size() * sizeof(uint32_t),
                                cudaMemcpyHostToDevice, e->stream), "table upload"))
        return LBM_ERR_CUDA;
    if (!e->list) {   // the members' non-plain cells beyond plain bounce-back (the step kernel updates those), concatenated
        size_t total = 0;
        for (lbm_handle* h : e->m) total += h->n_complex;
        if (total > 0xFFFFFFFFull) return LBM_ERR_UNSUPPORTED;
        if (total > 0) {
            if (e->cuda(cudaMalloc((void**)&e->list, total * sizeof(uint64_t)), "list alloc")) return LBM_ERR_OOM;
            size_t at = 0;
            for (size_t k = 0; k < e->m.size(); ++k) {
                const lbm_handle* h = e->m[k];
                if (!h->n_complex) continue;
                k_tag_cells<<<(unsigned)std::min<size_t>((h->n_complex + 255) / 256, 1024), 256, 0, e->stream>>>(
                    h->special, h->n_complex, (uint32_t)k, e->list + at);
                if (e->cuda(cudaGetLastError(), "list kernel")) return LBM_ERR_CUDA;
                at += h->n_complex;
            }
        }
        e->n_list = (uint32_t)total;
    }
    if (e->cuda(cudaStreamSynchronize(e->stream), "sync")) return LBM_ERR_CUDA;
    e->drop_graphs();
    e->keys.clear();
    for (const lbm_handle* h : e->m) e->keys.emplace_back(h);
    return LBM_OK;
}

// kernel launch of ensemble step number `s` (0-based since creation)
lbm_status launch(lbm_ensemble* e, int64_t s, cudaStream_t stream) {
    Launch L;
    L.block = e->variant == LBM_ENS_PAIRED ? dim3(32, e->warps, 1) : dim3(e->tile, 1, 1);
    L.grid = dim3(e->total_tiles, 1, 1);
    L.stream = stream;
    const int64_t t = e->t0[0] + s;
    const int scheme = !e->aa ? SCHEME_AB : ((t & 1) ? SCHEME_AA_LOC : SCHEME_AA_PP);
    const int parity = e->aa ? 0 : (int)(s & 1);
    const bool ch = e->layout == LBM_LAYOUT_CHUNKED;
    lbm_status st;
    if (e->variant == LBM_ENS_PAIRED)
        st = e->cuda(e->ks->ens_pair[ch ? 1 : 0](e->table, e->tile_member, parity, L), "paired ensemble kernel");
    else if (ch)
        st = e->cuda(e->ks->ens_ch[scheme](e->table, e->tile_member, parity, L), "ensemble kernel");
    else
        st = e->cuda(e->ks->ens[scheme][e->idx32 ? 1 : 0](e->table, e->tile_member, parity, L), "ensemble kernel");
    if (st != LBM_OK || e->n_list == 0) return st;
    Launch B;
    B.block = dim3(256, 1, 1);
    B.grid = dim3((e->n_list + 255) / 256, 1, 1);
    B.stream = stream;
    if (ch) return e->cuda(e->ks->ens_list_ch[scheme](e->table, e->list, e->n_list, parity, B), "ensemble list kernel");
    return e->cuda(e->ks->ens_list[scheme][e->idx32 ? 1 : 0](e->table, e->list, e->n_list, parity, B),
                   "ensemble list kernel");
}

lbm_status check_members(lbm_ensemble* e) {
    for (size_t k = 0; k < e->m.size(); ++k) {
        if (e->m[k]->sticky) return LBM_ERR_STATE;
        if (e->m[k]->t != e->t0[k] + e->s) {
            e->err = "a member was stepped or re-initialised outside the ensemble; create a new ensemble";
            return LBM_ERR_STATE;
        }
        if (k < e->keys.size() && !(MemberKey(e->m[k]) == e->keys[k])) {
            e->err = "a member's geometry, nodes, scheme or layout changed outside the ensemble; create a new ensemble";
            return LBM_ERR_STATE;
        }
    }
    return LBM_OK;
}

void advance_members(lbm_ensemble* e, int64_t n) {
    for (lbm_handle* h : e->m) {
        h->t += n;
        if (!h->aa() && (n & 1)) h->cur ^= 1;
    }
    e->s += n;
}

}  // namespace

extern "C" lbm_status lbm_ensemble_create(lbm_handle* const* members, int count, lbm_ensemble** out) {
    if (!members || count < 1 || !out) return LBM_ERR_ARG;
    *out = nullptr;
    lbm_handle* h0 = members[0];
    if (!h0 || h0->p.velset != LBM_D3Q19) return LBM_ERR_UNSUPPORTED;
    long long tiles_bound = 0;
    for (int k = 0; k < count; ++k) {
        lbm_handle* h = members[k];
        if (!h) return LBM_ERR_ARG;
        if (h->sticky) return LBM_ERR_STATE;
        if (h->p.velset != h0->p.velset || h->p.collision != h0->p.collision || h->p.storage != h0->p.storage ||
            h->p.arith != h0->p.arith || h->p.scheme != h0->p.scheme || !h->flags || (h->t & 1) != (h0->t & 1))
            return LBM_ERR_ARG;
        for (int j = 0; j < k; ++j)
            if (members[j] == h) return LBM_ERR_ARG;
        tiles_bound += (long long)h->N;   // at least one cell per tile
    }
    if (tiles_bound > 0x7FFFFFFFll) return LBM_ERR_UNSUPPORTED;
    // the ensemble kernels address the structure-of-arrays layout
    for (int k = 0; k < count; ++k)
        if (members[k]->chunked) {
            const lbm_status st = lbm_set_variant(members[k], LBM_VARIANT_GENERIC);
            if (st != LBM_OK) return st;
        }
    lbm_ensemble* e = new lbm_ensemble;
    e->m.assign(members, members + count);
    e->stream = h0->stream;
    e->ks = h0->ks;
    e->fp64 = h0->fp64();
    e->aa = h0->aa();
    for (lbm_handle* h : e->m) {
        e->t0.push_back(h->t);
        e->idx32 = e->idx32 && h->idx32();
        if (h->stream != e->stream &&
            std::find(e->member_streams.begin(), e->member_streams.end(), h->stream) == e->member_streams.end())
            e->member_streams.push_back(h->stream);
    }
    if (order_streams(e, true) != LBM_OK) {   // the members' geometry and fields are set
        lbm_ensemble_destroy(e);
        return LBM_ERR_CUDA;
    }
    if (cudaStreamCreateWithFlags(&e->capture, cudaStreamNonBlocking) != cudaSuccess) {
        delete e;
        return LBM_ERR_CUDA;
    }
    {   // which members have non-solid cells on a face (the paired kernel sends those through the per-cell path)
        int* dev = nullptr;
        if (cudaMalloc((void**)&dev, sizeof(int) * count) != cudaSuccess) {
            lbm_ensemble_destroy(e);
            return LBM_ERR_OOM;
        }
        cudaMemsetAsync(dev, 0, sizeof(int) * count, e->stream);
        for (int k = 0; k < count; ++k) {
            const lbm_handle* h = members[k];
            k_face_open<<<(unsigned)std::min<size_t>((h->N + 255) / 256, 1024), 256, 0, e->stream>>>(
                h->flags, h->p.nx, h->p.ny, h->p.nz, dev + k);
        }
        std::vector<int> host(count);
        const cudaError_t ce = cudaMemcpyAsync(host.data(), dev, sizeof(int) * count, cudaMemcpyDeviceToHost, e->stream);
        const cudaError_t se = cudaStreamSynchronize(e->stream);
        cudaFree(dev);
        if (ce != cudaSuccess || se != cudaSuccess) {
            lbm_ensemble_destroy(e);
            return LBM_ERR_CUDA;
        }
        e->open.assign(host.begin(), host.end());
    }
    const lbm_status st = upload_table(e);
    if (st != LBM_OK) {
        lbm_ensemble_destroy(e);
        return st;
    }
    *out = e;
    return LBM_OK;
}

extern "C" lbm_status lbm_ensemble_destroy(lbm_ensemble* e) {
    if (!e) return LBM_OK;
    // the ensemble's launches end before the members' streams touch their copies
    cudaStreamSynchronize(e->stream);
    // members on the chunked layout go back to the layout of their own settings
    if (e->layout == LBM_LAYOUT_CHUNKED)
        for (lbm_handle* h : e->m)
            if (h->force_chunked && !h->sticky) {
                h->force_chunked = false;
                lbm_internal_ensure_layout(h);
            }
    cudaStreamSynchronize(e->stream);
    e->drop_graphs();
    if (e->table) cudaFree(e->table);
    if (e->tile_member) cudaFree(e->tile_member);
    if (e->list) cudaFree(e->list);
    if (e->capture) cudaStreamDestroy(e->capture);
    if (e->order) cudaEventDestroy(e->order);
    delete e;
    return LBM_OK;
}

extern "C" lbm_status lbm_ensemble_step(lbm_ensemble* e, int64_t nsteps) {
    if (!e || nsteps < 0) return LBM_ERR_ARG;
    lbm_status st = check_members(e);
    if (st != LBM_OK) return st;
    if ((st = order_streams(e, true)) != LBM_OK) return st;
    int64_t done = 0;
    while (nsteps - done >= kGraphSteps) {
        const int key = (int)((e->aa ? e->t0[0] + e->s : e->s) & 1);
        if (!e->graph[key]) {
            cudaGraph_t g = nullptr;
            if (e->cuda(cudaStreamBeginCapture(e->capture, cudaStreamCaptureModeThreadLocal), "capture")) return LBM_ERR_CUDA;
            lbm_status cst = LBM_OK;
            for (int k = 0; k < kGraphSteps && cst == LBM_OK; ++k) cst = launch(e, e->s + k, e->capture);
            const cudaError_t ce = cudaStreamEndCapture(e->capture, &g);
            if (cst != LBM_OK) { if (g) cudaGraphDestroy(g); return cst; }
            if (e->cuda(ce, "end capture")) return LBM_ERR_CUDA;
            const cudaError_t ie = cudaGraphInstantiate(&e->graph[key], g, 0);
            cudaGraphDestroy(g);
            if (e->cuda(ie, "graph instantiate")) return LBM_ERR_CUDA;
        }
        if (e->cuda(cudaGraphLaunch(e->graph[key], e->stream), "graph launch")) return LBM_ERR_CUDA;
        advance_members(e, kGraphSteps);
        done += kGraphSteps;
    }
    for (; done < nsteps; ++done) {
        st = launch(e, e->s, e->stream);
        if (st != LBM_OK) return st;
        advance_members(e, 1);
    }
    return order_streams(e, false);
}

extern "C" lbm_status lbm_ensemble_step_each(lbm_ensemble* e, int64_t nsteps) {
    if (!e || nsteps < 0) return LBM_ERR_ARG;
    lbm_status st = check_members(e);
    if (st != LBM_OK) return st;
    if ((st = order_streams(e, true)) != LBM_OK) return st;
    for (int64_t k = 0; k < nsteps; ++k) {
        for (lbm_handle* h : e->m) {
            st = lbm_internal_step(h, e->stream);   // advances h's counters
            if (st != LBM_OK) return st;
        }
        e->s += 1;
    }
    return order_streams(e, false);
}

extern "C" lbm_status lbm_ensemble_set_block(lbm_ensemble* e, int bx, int by) {
    if (!e || bx < 32 || by != 1 || bx > 256 || (bx % 32) != 0) return LBM_ERR_ARG;
    lbm_status st = check_members(e);
    if (st != LBM_OK) return st;
    e->tile = bx;
    return upload_table(e);
}

namespace {
bool pair_ok(const lbm_ensemble* e) { return e->ks->ens_pair[0] && !e->aa && e->idx32; }
bool chunked_ok(const lbm_ensemble* e) { return e->ks->ens_ch[0] && e->idx32; }
}  // namespace

extern "C" lbm_status lbm_ensemble_set_layout(lbm_ensemble* e, int layout) {
    if (!e || (layout != LBM_LAYOUT_SOA && layout != LBM_LAYOUT_CHUNKED)) return LBM_ERR_ARG;
    lbm_status st = check_members(e);
    if (st != LBM_OK) return st;
    if (layout == LBM_LAYOUT_CHUNKED && !chunked_ok(e)) {
        e->err = "the chunked member layout needs 16-bit storage with FP32 arithmetic, SRT or TRT collision and "
                 "q N < 2^32 for every member";
        return LBM_ERR_UNSUPPORTED;
    }
    if (layout == e->layout) return LBM_OK;
    for (lbm_handle* h : e->m) {
        h->force_chunked = layout == LBM_LAYOUT_CHUNKED;
        if ((st = lbm_internal_ensure_layout(h)) != LBM_OK) {
            e->err = std::string("layout change: ") + lbm_last_error(h);
            return st;
        }
    }
    e->layout = layout;
    return upload_table(e);
}

extern "C" int lbm_ensemble_get_layout(const lbm_ensemble* e) { return e ? e->layout : -1; }

extern "C" lbm_status lbm_ensemble_set_variant(lbm_ensemble* e, int variant, int warps) {
    if (!e) return LBM_ERR_ARG;
    if (variant != LBM_ENS_PER_CELL && variant != LBM_ENS_PAIRED) return LBM_ERR_ARG;
    if (variant == LBM_ENS_PAIRED && (warps < 1 || warps > 4)) return LBM_ERR_ARG;
    lbm_status st = check_members(e);
    if (st != LBM_OK) return st;
    if (variant == LBM_ENS_PAIRED && !pair_ok(e)) {
        e->err = "the paired ensemble kernel needs A-B streaming, FP16 or FP16S storage with FP32 arithmetic, "
                 "SRT or TRT collision and q N < 2^32 for every member";
        return LBM_ERR_UNSUPPORTED;
    }
    e->variant = variant;
    if (variant == LBM_ENS_PAIRED) e->warps = warps;
    return upload_table(e);
}

extern "C" int lbm_ensemble_get_variant(const lbm_ensemble* e) { return e ? e->variant : -1; }

namespace {

// One configuration of the ensemble launch: the per-cell kernel with a tile
// size, or the paired kernel with warps per tile.
struct EnsConfig {
    int variant, size;
};

// times every configuration that applies to the current scheme; returns the best
lbm_status time_configs(lbm_ensemble* e, int trial_steps, float* best_ms, EnsConfig* best) {
    static const int tiles[] = {256, 128, 64, 192, 96};
    static const int warps[] = {4, 2, 1};
    std::vector<EnsConfig> cfg;
    for (int t : tiles) cfg.push_back({LBM_ENS_PER_CELL, t});
    if (pair_ok(e))
        for (int w : warps) cfg.push_back({LBM_ENS_PAIRED, w});
    cudaEvent_t ev[2];
    if (e->cuda(cudaEventCreate(&ev[0]), "event") || e->cuda(cudaEventCreate(&ev[1]), "event")) return LBM_ERR_CUDA;
    lbm_status st = LBM_OK;
    *best_ms = INFINITY;
    for (const EnsConfig& c : cfg) {
        st = c.variant == LBM_ENS_PAIRED ? lbm_ensemble_set_variant(e, LBM_ENS_PAIRED, c.size)
                                         : lbm_ensemble_set_variant(e, LBM_ENS_PER_CELL, 0);
        if (st == LBM_OK && c.variant == LBM_ENS_PER_CELL) st = lbm_ensemble_set_block(e, c.size, 1);
        if (st != LBM_OK) break;
        st = lbm_ensemble_step(e, 2);   // warm-up
        if (st != LBM_OK) break;
        cudaEventRecord(ev[0], e->stream);
        st = lbm_ensemble_step(e, trial_steps);
        if (st != LBM_OK) break;
        cudaEventRecord(ev[1], e->stream);
        if (e->cuda(cudaEventSynchronize(ev[1]), "event sync")) { st = LBM_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (ms < *best_ms) { *best_ms = ms; *best = c; }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    return st;
}

lbm_status apply_config(lbm_ensemble* e, const EnsConfig& c) {
    if (c.variant == LBM_ENS_PAIRED) return lbm_ensemble_set_variant(e, LBM_ENS_PAIRED, c.size);
    const lbm_status st = lbm_ensemble_set_variant(e, LBM_ENS_PER_CELL, 0);
    return st != LBM_OK ? st : lbm_ensemble_set_block(e, c.size, 1);
}

// converts every member (lbm_set_scheme) and rebuilds the ensemble's tables
lbm_status switch_scheme(lbm_ensemble* e, int scheme) {
    const int back = e->aa ? LBM_STREAM_AA : LBM_STREAM_AB;
    for (size_t k = 0; k < e->m.size(); ++k) {
        const lbm_status st = lbm_set_scheme(e->m[k], scheme);
        if (st != LBM_OK) {   // e.g. no memory for A-B copies: undo the members switched so far
            e->err = std::string("scheme switch: ") + lbm_last_error(e->m[k]);
            for (size_t j = 0; j < k; ++j) lbm_set_scheme(e->m[j], back);
            // the members switched back hold new copies: tables from them
            const std::string why = e->err;
            if (upload_table(e) == LBM_OK) e->err = why;
            return st;
        }
    }
    e->aa = scheme == LBM_STREAM_AA;
    for (lbm_handle* h : e->m) e->idx32 = e->idx32 && h->idx32();
    return upload_table(e);
}

bool can_use_aa(const lbm_ensemble* e) {
    for (const lbm_handle* h : e->m)
        if (h->has_open_boundaries) return false;
    return true;
}

}  // namespace

extern "C" lbm_status lbm_ensemble_autotune(lbm_ensemble* e, int trial_steps, int* bx_out, int* by_out) {
    if (!e || trial_steps < 1) return LBM_ERR_ARG;
    lbm_status st = check_members(e);
    if (st != LBM_OK) return st;
    trial_steps += trial_steps & 1;       // whole A-A step pairs: the scheme may change between trials
    struct Best {
        float ms = INFINITY;
        int layout = LBM_LAYOUT_SOA, scheme = LBM_STREAM_AB;
        EnsConfig c{LBM_ENS_PER_CELL, 256};
    } best;
    const int scheme0 = e->aa ? LBM_STREAM_AA : LBM_STREAM_AB;
    const int scheme1 = e->aa ? LBM_STREAM_AB : LBM_STREAM_AA;
    // the other streaming scheme, where every member allows it (A-A: no
    // outflow or free-slip cells) and the memory for A-B copies is there
    const bool other = (scheme1 == LBM_STREAM_AB || can_use_aa(e)) && ((e->t0[0] + e->s) & 1) == 0;
    std::vector<int> layouts{e->layout};
    if (chunked_ok(e)) layouts.push_back(e->layout == LBM_LAYOUT_SOA ? LBM_LAYOUT_CHUNKED : LBM_LAYOUT_SOA);
    for (int layout : layouts) {
        if ((st = lbm_ensemble_set_variant(e, LBM_ENS_PER_CELL, 0)) != LBM_OK) return st;
        if ((st = lbm_ensemble_set_layout(e, layout)) != LBM_OK) return st;
        for (int pass = 0; pass < (other ? 2 : 1); ++pass) {
            const int scheme = pass == 0 ? scheme0 : scheme1;
            if (pass == 1) {
                if ((st = lbm_ensemble_set_variant(e, LBM_ENS_PER_CELL, 0)) != LBM_OK) return st;
                if (switch_scheme(e, scheme1) != LBM_OK) break;   // e.g. no memory for A-B copies
            }
            float ms = INFINITY;
            EnsConfig c{LBM_ENS_PER_CELL, e->tile};
            if ((st = time_configs(e, trial_steps, &ms, &c)) != LBM_OK) return st;
            if (ms < best.ms) {
                best.ms = ms;
                best.layout = layout;
                best.scheme = scheme;
                best.c = c;
            }
            if (pass == 1) {
                if ((st = lbm_ensemble_set_variant(e, LBM_ENS_PER_CELL, 0)) != LBM_OK) return st;
                if ((st = switch_scheme(e, scheme0)) != LBM_OK) return st;
            }
        }
    }
    if ((st = lbm_ensemble_set_variant(e, LBM_ENS_PER_CELL, 0)) != LBM_OK) return st;
    if ((st = lbm_ensemble_set_layout(e, best.layout)) != LBM_OK) return st;
    if (best.scheme != scheme0 && (st = switch_scheme(e, best.scheme)) != LBM_OK) return st;
    st = apply_config(e, best.c);
    if (bx_out) *bx_out = best.c.variant == LBM_ENS_PAIRED ? 64 * best.c.size : best.c.size;
    if (by_out) *by_out = best.c.variant == LBM_ENS_PAIRED ? best.c.size : 1;
    return st;
}

extern "C" int lbm_ensemble_scheme(const lbm_ensemble* e) {
    return e ? (e->aa ? LBM_STREAM_AA : LBM_STREAM_AB) : -1;
}

extern "C" const char* lbm_ensemble_last_error(const lbm_ensemble* e) { return e ? e->err.c_str() : "null ensemble"; }
