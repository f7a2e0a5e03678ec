/*
 * lbm.h -- C ABI of the GB300 (sm_103a) mixed-precision lattice Boltzmann library.
 *
 * The library implements the fused stream-collide step of Lehmann et al.,
 * "On the accuracy and performance of the lattice Boltzmann method with
 * 64-bit, 32-bit and novel 16-bit number formats" (arXiv 2112.08926):
 * populations (DDFs) are stored shifted (Sec. 2.2) in FP64, FP32 or one of
 * the 16-bit formats of Sec. 3, while the collision runs in FP32 (or FP64)
 * registers.  Every step of the path runs in CUDA kernels; the host code only
 * validates arguments, moves data and launches.
 *
 * Conventions shared by every entry point
 *   - Cell index n = x + nx*(y + ny*z), x fastest (the paper's appendix core
 *     uses the same linearisation).
 *   - Host arrays belong to the caller and are read or written before the
 *     call returns.  Device memory is owned by the handle and obtained
 *     through the lbm_allocator given at creation (cudaMalloc if NULL).
 *   - Every call returns an lbm_status; nothing aborts or traps.  After a
 *     CUDA error the handle is poisoned: later calls return LBM_ERR_STATE and
 *     lbm_last_error() describes the first failure.
 *   - Velocity-set directions: 0 is rest, 2k-1 and 2k are opposite; D3Q19 in
 *     the order of the paper's D3Q19 core (+x -x +y -y +z -z, ++0 --0, +0+
 *     -0-, 0++ 0--, +-0 -+0, +0- -0+, 0+- 0-+); D3Q27 appends +++ ---, ++-
 *     --+, +-+ -+-, -++ +--; D2Q9 is 0, +x -x +y -y, ++ --, +- -+.
 *   - Populations are stored population-major (structure of arrays,
 *     f[i*N + n]) or in the chunked layout (LBM_LAYOUT_CHUNKED below); q*N
 *     codes per copy either way.  lbm_get_f / lbm_set_f always use the
 *     structure-of-arrays order.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,          /* invalid argument (reason in lbm_last_error) */
    LBM_ERR_OOM = 2,          /* the allocator returned NULL */
    LBM_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    LBM_ERR_UNSUPPORTED = 4,  /* valid but unsupported combination */
    LBM_ERR_DIVERGED = 5,     /* FP64 mass check found a non-finite value */
    LBM_ERR_TIMEOUT = 6,      /* a bounded device-side wait ran out */
    LBM_ERR_STATE = 7         /* handle poisoned by an earlier CUDA error, or a call that the
                                 object's state does not allow (see the calls) */
} lbm_status;

/* velocity sets (Sec. 2.1; D3Q19 main, D2Q9 and D3Q27 variants) */
enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1, LBM_D3Q27 = 2 };
/* collision operators: single- and two-relaxation-time (Sec. 2.1), and the
 * D3Q19 multiple-relaxation-time operator of the Sec. 5 roofline, which the
 * paper does not define: the orthogonal moment basis and relaxation rates of
 * d'Humieres et al. (2002), shear and conserved moments relaxed with 1/tau,
 * the second-order equilibrium and Guo source of the other operators */
enum { LBM_SRT = 0, LBM_TRT = 1, LBM_MRT = 2 };
/* storage formats of the populations (Sec. 3, Table 2).  P16_0 / P16_1 are
 * the posit formats of Sec. 3.2 without the 2^7 scaling. */
enum {
    LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16 = 2, LBM_FP16S = 3, LBM_FP16C = 4,
    LBM_P16_0S = 5, LBM_P16_1S = 6, LBM_P16_2C = 7, LBM_P16_0 = 8, LBM_P16_1 = 9
};
/* arithmetic precision of the collision (the "FPa" of the paper's "FPa/FPs") */
enum { LBM_ARITH_FP32 = 0, LBM_ARITH_FP64 = 1 };
/* streaming scheme: one-step pull with two copies (A-B, Sec. 5) or the
 * in-place A-A scheme with one copy (Sec. 1 "any swap algorithm").  AUTO (a
 * creation parameter only): A-B when both copies fit in the device's free
 * memory with a 10% margin, else A-A; lbm_autotune then also times the
 * other scheme where the lattice allows it.  lbm_get_info reports the
 * scheme in use. */
enum { LBM_STREAM_AB = 0, LBM_STREAM_AA = 1, LBM_STREAM_AUTO = 2 };

/* cell flag bits (one byte per cell) */
#define LBM_FLUID        0x00u
#define LBM_WALL         0x01u  /* solid: mid-grid bounce-back (Sec. 4.1) */
#define LBM_MOVING       0x02u  /* with WALL: moving bounce-back (Sec. 4.4), velocity in node_u */
#define LBM_EQ           0x04u  /* equilibrium boundary node (Sec. 4.3): node_rho, node_u */
#define LBM_OUTFLOW      0x08u  /* zero-gradient outflow: copies the -x neighbour's inflow */
#define LBM_FREESLIP     0x10u  /* with WALL: specular wall, normal axis in bits 5-6 */
#define LBM_FREESLIP_AXIS(a) ((uint8_t)(LBM_WALL | LBM_FREESLIP | ((a) << 5)))

typedef struct {
    int nx, ny, nz;     /* lattice size; D2Q9 requires nz == 1 */
    int velset;         /* LBM_D2Q9, LBM_D3Q19, LBM_D3Q27 */
    int collision;      /* LBM_SRT, LBM_TRT, LBM_MRT (D3Q19; FP64/FP64, FP32/FP32,
                           FP32/FP16S and FP32/FP16C; others LBM_ERR_UNSUPPORTED) */
    int storage;        /* LBM_FP64 .. LBM_P16_1 */
    int arith;          /* LBM_ARITH_FP32; LBM_ARITH_FP64 only with FP64/FP32 storage */
    int scheme;         /* LBM_STREAM_AB, LBM_STREAM_AA, LBM_STREAM_AUTO */
    double tau;         /* relaxation time (> 0.5); omega = 1/tau (appendix, SRT) */
    double trt_lambda;  /* TRT magic parameter (tau+ - 1/2)(tau- - 1/2), e.g. 3/16 */
    double force[3];    /* Guo body force per volume (Sec. 4.1); D2Q9 ignores z */
    int no_ddf_shifting; /* 0 (default): populations stored shifted, f - w (Sec. 2.2);
                            1: stored unshifted, the ablation of the paper's dashed
                            curves (appendix, "without DDF-shifting") */
} lbm_params;

typedef struct {
    /* Returns device memory of `bytes` bytes (256-byte aligned) or NULL. */
    void* (*alloc)(size_t bytes, void* ctx);
    void (*release)(void* ptr, void* ctx);
    void* ctx;
} lbm_allocator;

typedef struct lbm_handle lbm_handle;

/* Create a lattice.  Allocates the population copies (one for A-A, two for
 * A-B), flags and boundary-node arrays, and scratch.  All cells start as
 * fluid at rest (rho = 1, u = 0: zero shifted populations).  cuda_stream is a
 * cudaStream_t; NULL selects the legacy default stream.
 * Errors: LBM_ERR_ARG (bad sizes/enums/tau), LBM_ERR_UNSUPPORTED (FP64
 * arithmetic with 16-bit storage, more than 2^31 cells), LBM_ERR_OOM,
 * LBM_ERR_CUDA. */
lbm_status lbm_create(const lbm_params* params, const lbm_allocator* allocator,
                      void* cuda_stream, lbm_handle** out);

/* Release every device allocation; NULL is accepted. */
lbm_status lbm_destroy(lbm_handle* h);

/* Cell types and boundary data, host arrays of N = nx*ny*nz cells.
 * flags: N bytes (NULL: every cell fluid, fully periodic -- the flag-free
 * kernel of the paper's periodic benchmark box, Sec. 5); node_u: 3*N floats
 * component-major (ux[N], uy[N], uz[N]; wall velocity of MOVING cells, state
 * of EQ cells) or NULL (zero); node_rho: N floats (EQ density) or NULL (1).
 * The populations of cells that are solid in the new geometry are set to
 * zero.  The first call with flags allocates, through the lattice's
 * allocator, the flag bytes (N), a 32-bit wall mask per cell (4 N bytes:
 * the directions whose upstream cell is solid, read by the fast kernels
 * for cells that only bounce back), the node arrays the flags need and
 * the list of boundary cells.  With A-A streaming, OUTFLOW and FREESLIP cells give
 * LBM_ERR_UNSUPPORTED.  Invalid bit combinations, and OUTFLOW cells whose
 * -x neighbour is solid (an outflow cell pulls as if it sat there), give
 * LBM_ERR_ARG. */
lbm_status lbm_set_geometry(lbm_handle* h, const uint8_t* flags, const float* node_u,
                            const float* node_rho);

/* Boundary-node data of listed cells only, for lattices whose boundary is a
 * small part of the domain (a 1024^3 cavity has 10^6 lid cells among 10^9):
 * the wall velocity of MOVING cells (Sec. 4.4) and the state of EQ cells
 * (Sec. 4.3) without full-size host arrays.  cells: `count` distinct indices
 * in [0, N); node_u: 3*count floats, component-major (ux[count], uy[count],
 * uz[count]), or NULL to leave velocities unchanged; node_rho: count floats
 * or NULL.  Cells not listed keep their values (zero velocity, unit density
 * after lbm_set_geometry without node arrays).  Needs flags set by
 * lbm_set_geometry.  Takes effect from the next step.  Errors: LBM_ERR_ARG
 * (no flags, index out of range, an index listed twice), LBM_ERR_OOM. */
lbm_status lbm_set_nodes(lbm_handle* h, int64_t count, const int64_t* cells, const float* node_u,
                         const float* node_rho);

/* Initialise every non-solid cell with the shifted equilibrium (Sec. 2.2;
 * the plain one with no_ddf_shifting) of the given density and velocity (host arrays of N doubles; NULL means
 * rho = 1 / u = 0), converted to the arithmetic precision first; solid cells
 * get zero populations.  Resets the step counter to 0. */
lbm_status lbm_set_rho_u(lbm_handle* h, const double* rho, const double* ux,
                         const double* uy, const double* uz);

/* Advance nsteps time steps (each: pull streaming + collision, appendix
 * "LBM equations in a nutshell", fused in one kernel).  Asynchronous on the
 * handle's stream.  On lattices of up to 2^23 cells, calls of 64 steps or
 * more replay runs of 32 steps from a CUDA graph, captured on a private
 * stream and kept until a call changes what a step launches; the results
 * are those of one launch per step. */
lbm_status lbm_step(lbm_handle* h, int64_t nsteps);

/* Divergence check inside lbm_step (off by default): after every `every`
 * steps of the lattice's step counter, lbm_step runs the FP64 reduction of
 * lbm_reduce and returns LBM_ERR_DIVERGED, with the step reached in
 * lbm_last_error, when the mass or the kinetic energy is not finite or the
 * mass has drifted from its value when the check was set by more than
 * mass_tol relative (mass_tol <= 0: finiteness only).  The populations stay
 * as they are (the handle is not poisoned); each check synchronises the
 * stream, and the steps in between keep their graphs.  every = 0 switches
 * the check off.  Errors: LBM_ERR_ARG (every < 0 or mass_tol not finite),
 * LBM_ERR_DIVERGED if the state is already non-finite when the check is set. */
lbm_status lbm_set_divergence_check(lbm_handle* h, int64_t every, double mass_tol);

/* Density and velocity of every cell from the streamed populations: rho =
 * (sum f_i) + 1 (Sec. 2.2), u = (sum c_i f_i + F/2)/rho (not clamped).
 * EQ cells report their node state, solid cells rho = 1, u = 0.  Host arrays
 * of N doubles (any may be NULL).  Synchronises the stream. */
lbm_status lbm_get_rho_u(lbm_handle* h, double* rho, double* ux, double* uy, double* uz);

/* lbm_get_rho_u without any device allocation (the paper has no counterpart;
 * this is a service for callers that cannot allocate).  lbm_get_rho_u takes
 * a staging buffer from the lattice's allocator for the length of the call;
 * a caller whose device memory is already fully used by the simulation, or
 * that must not call cudaMalloc (it blocks the device and competes with a
 * framework's memory pool), can use this entry point instead.  It writes the
 * same values, staging through one fixed array of 2^20 doubles (8 MiB) that
 * the library places on every GPU it is used on; the array stays until the
 * process exits.  Limit: nx*ny <= 262144 cells (four doubles per cell of one
 * xy-plane must fit); larger planes give LBM_ERR_UNSUPPORTED with the reason
 * in lbm_last_error.
 * Set-up: the array's device address is looked up (cudaGetSymbolAddress,
 * which also makes the CUDA runtime place the array) when the first lattice
 * on a device is created, with that device current, so the memory is taken
 * before a simulation fills the GPU and before any stream capture.  If that
 * look-up failed, this call returns LBM_ERR_UNSUPPORTED and leaves the
 * lattice usable.  The kernels it launches are loaded at their first launch
 * in the process, like every other kernel of the library.
 * All calls share the array: calls whose work overlaps on the GPU (lattices
 * on different streams read out at the same time) race and must be
 * serialised by the caller.  Every chunk is written completely before it is
 * read, so no state carries over between calls.  Like lbm_get_rho_u it
 * reports LBM_ERR_TIMEOUT if a kernel of an earlier step gave up a bounded
 * wait.  Host arrays as for lbm_get_rho_u; synchronises the lattice's
 * stream. */
lbm_status lbm_get_rho_u_static(lbm_handle* h, double* rho, double* ux, double* uy, double* uz);

/* Streamed populations f_i(x) (shifted unless no_ddf_shifting, decoded,
 * exactly as the next collision reads them) into a host array of q*N doubles; solid cells 0. */
lbm_status lbm_get_f(lbm_handle* h, double* f);

/* Point probes: the streamed populations (as lbm_get_f) of `count` listed
 * cells into f, population-major (f[i*count + k] for the k-th listed cell),
 * and the density and velocity (as lbm_get_rho_u) of listed cells into
 * arrays of `count` doubles (any may be NULL).  cells: host array of indices
 * in [0, N), repeats allowed.  Errors: LBM_ERR_ARG (index out of range,
 * NULL arrays), LBM_ERR_OOM.  Synchronise the stream. */
lbm_status lbm_get_f_cells(lbm_handle* h, int64_t count, const int64_t* cells, double* f);
lbm_status lbm_get_rho_u_cells(lbm_handle* h, int64_t count, const int64_t* cells, double* rho, double* ux,
                               double* uy, double* uz);

/* Overwrite the post-collision populations (what every cell streams out at
 * the next step) from a host array of q*N doubles, encoded to the storage
 * format.  Resets the step counter to 0. */
lbm_status lbm_set_f(lbm_handle* h, const double* f);

/* FP64 sums over non-solid cells of rho and rho |u|^2 / 2 (u with the Guo
 * half-force), computed on the device.  Returns LBM_ERR_DIVERGED if either
 * sum is not finite.  Synchronises the stream. */
lbm_status lbm_reduce(lbm_handle* h, double* mass, double* kinetic_energy);

/* memory layout of the populations: structure of arrays f[i*N + n], or the
 * chunked layout of lattices with 16-bit storage, FP32 arithmetic and nx a
 * multiple of 64 (A-B or A-A, with or without flags; D3Q27 only with FP16 or
 * FP16S; chosen by LBM_VARIANT_AUTO / _PAIRED): the cells of each row are
 * cut into chunks of 64, and chunk c = n/64 holds its q populations one
 * after the other, element ((n/64)*q + i)*64 + n%64. */
enum { LBM_LAYOUT_SOA = 0, LBM_LAYOUT_CHUNKED = 1 };

typedef struct {
    int q;                    /* populations per cell */
    int64_t cells;            /* N */
    int64_t step;             /* steps taken since the last initialisation */
    int bytes_per_population; /* 8, 4 or 2 */
    int has_flags;            /* 0: flag-free periodic kernel */
    size_t device_bytes;      /* bytes held on the device */
    void* ddf[2];             /* device population copies (ddf[1] NULL for A-A) */
    int layout;               /* LBM_LAYOUT_SOA or LBM_LAYOUT_CHUNKED */
    int scheme;               /* LBM_STREAM_AB or LBM_STREAM_AA (in use) */
} lbm_info;

lbm_status lbm_get_info(const lbm_handle* h, lbm_info* info);

/* Thread-block shape of the stream-collide launches (threads along x and y;
 * bx*by a multiple of 32, at most 1024).  Default 128 x 2. */
lbm_status lbm_set_block(lbm_handle* h, int bx, int by);

/* Stream-collide kernel variants; all give bit-for-bit the same result.
 *   GENERIC  one cell per thread, every lattice and boundary kind;
 *   PAIRED   two x-neighbouring cells per thread, populations moved as
 *            32-bit pairs of codes, 16-bit storage and FP32 arithmetic:
 *            with nx a multiple of 64 on the chunked layout
 *            (LBM_LAYOUT_CHUNKED; A-B or A-A, with or without flags),
 *            every warp moving whole 128-byte lines at compile-time
 *            offsets; otherwise on the structure-of-arrays layout for
 *            flag-free A-B lattices with even nx, q*N < 2^32 and a block
 *            width that is a multiple of 32;
 *   STAGED   source rows prefetched into shared memory by bulk copies
 *            several tiles ahead (flag-free A-B D3Q19 lattices, FP32
 *            arithmetic, nx of 128, 256 or 512); a copy wait that runs out
 *            (about a second) makes the next synchronising call return
 *            LBM_ERR_TIMEOUT;
 *   AUTO     (default) PAIRED where it applies, else GENERIC.
 * A requested variant that does not apply falls back to GENERIC.  Switching
 * variant, or setting flags, converts the stored populations between the
 * layouts (no change in values). */
enum { LBM_VARIANT_AUTO = 0, LBM_VARIANT_GENERIC = 1, LBM_VARIANT_STAGED = 2, LBM_VARIANT_PAIRED = 3 };
lbm_status lbm_set_variant(lbm_handle* h, int variant);
/* The variant lbm_step launches for h now (LBM_VARIANT_GENERIC, _STAGED or
 * _PAIRED), or -1 for a NULL handle. */
int lbm_get_variant(const lbm_handle* h);

/* Switch the streaming scheme of a live lattice (LBM_STREAM_AB or _AA)
 * without changing a value: after an even number of steps the A-B state
 * and the A-A state differ only by a swap of opposite slots.  AB -> AA
 * releases the second population copy (half the memory); AA -> AB
 * allocates it.  Errors: LBM_ERR_STATE after an odd number of steps,
 * LBM_ERR_UNSUPPORTED for A-A with OUTFLOW or FREESLIP cells, LBM_ERR_OOM. */
lbm_status lbm_set_scheme(lbm_handle* h, int scheme);

/* Times, over trial_steps steps each, the stream-collide kernel variants
 * that apply to the lattice -- GENERIC on the structure-of-arrays layout,
 * PAIRED (on the chunked layout where nx is a multiple of 64), STAGED -- and
 * keeps the fastest (its layout with it; query it with lbm_get_variant);
 * then, for the kernels that take one (GENERIC, PAIRED on the structure of
 * arrays), the thread-block shape, returned in *bx, *by; for a lattice created
 * with LBM_STREAM_AUTO, first the streaming scheme (A-B against in-place A-A,
 * switched with lbm_set_scheme where the step count is even, the lattice
 * has no OUTFLOW or FREESLIP cells and memory for the second copy is there).
 * Every choice gives the same values; the trial steps advance the lattice.
 * Otherwise the scheme stays as it is.  Trial runs of 64 steps or more
 * include one CUDA-graph capture (see lbm_step). */
lbm_status lbm_autotune(lbm_handle* h, int trial_steps, int* bx, int* by);

/* Self-test of the failure path (the paper has no counterpart): launches
 * one kernel whose bounded wait, on an mbarrier that nothing arrives on,
 * runs out after about a second, as a bulk copy that never lands would in
 * the STAGED kernel.  Returns LBM_ERR_TIMEOUT; the handle is then poisoned
 * exactly as after a real timeout (later calls give LBM_ERR_STATE) while the
 * CUDA context stays usable for other handles.  No fault, trap or hang. */
lbm_status lbm_selftest_wait_timeout(lbm_handle* h);

const char* lbm_last_error(const lbm_handle* h);
const char* lbm_status_string(lbm_status s);

/* ---- storage codecs as device-array kernels (the formats of Sec. 3) ------- */
/* x_dev: n floats, out_dev: n 16-bit codes; storage must be a 16-bit format.
 * Device pointers, asynchronous on cuda_stream. */
lbm_status lbm_codec_encode(int storage, const float* x_dev, uint16_t* out_dev, int64_t n,
                            void* cuda_stream);
lbm_status lbm_codec_decode(int storage, const uint16_t* c_dev, float* out_dev, int64_t n,
                            void* cuda_stream);
/* Encode the floats whose bit patterns are first, first+1, ..., first+n-1. */
lbm_status lbm_codec_encode_bits(int storage, uint32_t first, int64_t n, uint16_t* out_dev,
                                 void* cuda_stream);
/* The same through the table-driven encoder that the paired stream-collide
 * kernel uses for the posit formats (one fused multiply-add per value from a
 * per-exponent table held in shared memory); it gives the same codes as
 * lbm_codec_encode_bits.  Posit formats only (LBM_ERR_UNSUPPORTED otherwise). */
lbm_status lbm_codec_encode_bits_table(int storage, uint32_t first, int64_t n, uint16_t* out_dev,
                                       void* cuda_stream);

/* ---- ensembles: many independent lattices advanced by one launch per step -- */
typedef struct lbm_ensemble lbm_ensemble;

/* Group `count` D3Q19 handles that share collision, storage, arith and
 * scheme (LBM_ERR_ARG otherwise; other velocity sets LBM_ERR_UNSUPPORTED),
 * have flags set and the same step parity.  The members keep their own data;
 * the ensemble adds a device descriptor table and a per-tile member table.
 * All launches go to the first member's stream; where members have other
 * streams, each ensemble call first makes that stream wait (by events, the
 * host does not block) for the work already queued on theirs, and a step
 * makes their streams wait for its launches, so member calls before and
 * after ensemble steps stay in order. */
lbm_status lbm_ensemble_create(lbm_handle* const* members, int count, lbm_ensemble** out);
/* Advance every member nsteps steps: per step one launch over the plain
 * cells of all members and one over the listed boundary cells of all
 * members, replayed from a CUDA graph of up to 64 steps.  Every ensemble
 * call returns LBM_ERR_STATE (with lbm_ensemble_last_error) when a member
 * was stepped, re-initialised, given a new geometry or nodes, or switched
 * to another scheme or layout outside the ensemble since its tables were
 * built, or when a member handle is poisoned; create a new ensemble then. */
lbm_status lbm_ensemble_step(lbm_ensemble* e, int64_t nsteps);
/* Same result, member by member (two launches per member per step: the
 * baseline). */
lbm_status lbm_ensemble_step_each(lbm_ensemble* e, int64_t nsteps);
/* Cells per tile (thread block) of the ensemble launch: bx a multiple of 32
 * in [32, 256], by must be 1 (tiles are runs of consecutive cells). */
lbm_status lbm_ensemble_set_block(lbm_ensemble* e, int bx, int by);
/* Kernel of the ensemble's plain cells.
 *   PER_CELL  one cell per thread, tiles of lbm_ensemble_set_block cells,
 *             every scheme, storage format and collision (the default);
 *   PAIRED    two cells per thread, one warp per run of 64 consecutive cells
 *             of a member, every population moved as 32-bit pairs of codes
 *             (A-B, FP16 or FP16S storage with FP32 arithmetic, SRT or TRT,
 *             q N < 2^32 for every member); `warps` (1..4) runs per tile.
 *             Cells on the faces of members with non-solid face cells take
 *             the per-cell path inside the same launch.
 * Both give bit for bit the same populations.  Errors: LBM_ERR_ARG,
 * LBM_ERR_UNSUPPORTED (PAIRED where it does not apply). */
enum { LBM_ENS_PER_CELL = 0, LBM_ENS_PAIRED = 1 };
lbm_status lbm_ensemble_set_variant(lbm_ensemble* e, int variant, int warps);
int lbm_ensemble_get_variant(const lbm_ensemble* e);
/* Layout of the members' populations: LBM_LAYOUT_SOA (the default) or
 * LBM_LAYOUT_CHUNKED, the array of structures of arrays of chunks of 64
 * consecutive cells of the member's linear cell index (any nx; 16-bit
 * storage, FP32 arithmetic, SRT or TRT, q N < 2^32).  The members are
 * converted in place (no change in values); stepped on their own (also by
 * lbm_ensemble_step_each) they use kernels with the same addressing.
 * Destroying the ensemble returns them to the layout of their own settings.
 * Both kernels of lbm_ensemble_set_variant take either layout.  Errors:
 * LBM_ERR_ARG, LBM_ERR_UNSUPPORTED, LBM_ERR_OOM (A-A members convert through
 * a transient copy). */
lbm_status lbm_ensemble_set_layout(lbm_ensemble* e, int layout);
int lbm_ensemble_get_layout(const lbm_ensemble* e);
/* Picks the members' layout, the kernel, its tile and the streaming scheme:
 * for each layout that applies (structure of arrays; chunked) times
 * trial_steps steps (rounded up to even) for every tile size of the per-cell
 * kernel and, where it applies, every tile of the paired kernel; then, where
 * every member allows it (A-A: no OUTFLOW or FREESLIP cells; memory for the
 * A-B copies) and the step count is even, converts all members to the other
 * scheme (lbm_set_scheme) and times again; keeps the fastest combination.  *bx
 * receives the cells per tile, *by 1 for the per-cell kernel or the warps per
 * tile of the paired one.  The trial steps are real steps (two warm-up steps
 * per configuration on top).  Results do not depend on any of the choices. */
lbm_status lbm_ensemble_autotune(lbm_ensemble* e, int trial_steps, int* bx, int* by);
/* The streaming scheme the ensemble's members use now (-1 for NULL). */
int lbm_ensemble_scheme(const lbm_ensemble* e);
lbm_status lbm_ensemble_destroy(lbm_ensemble* e);
const char* lbm_ensemble_last_error(const lbm_ensemble* e);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
