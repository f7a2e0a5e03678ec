/*
 * CPU ORACLE for the mixed-precision lattice Boltzmann stream-collide step of
 * Lehmann et al., "On the accuracy and performance of the lattice Boltzmann
 * method with 64-bit, 32-bit and novel 16-bit number formats" (arXiv 2112.08926).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is a plain, slow, obviously correct
 * restatement of the paper's method.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant generator with the CUDA library under
 * paper_2112_08926_gb300/, and it never calls into it.
 *
 * Contents
 *   - number codecs for every storage format (Sec. 3, Table 2, Fig. 2);
 *   - an A-B pull lattice Boltzmann solver (appendix "LBM equations in a
 *     nutshell", Eqs. 1-4 and their shifted forms) for D2Q9, D3Q19 and D3Q27,
 *     SRT and TRT collision, half-way / moving bounce-back, equilibrium nodes,
 *     zero-gradient outflow, free-slip walls and Guo forcing.
 *
 * Arithmetic modes (see ORC_ARITH_*):
 *   DEF64  the plain textbook definition in FP64 with FP64 storage;
 *   ORD32  FP32 arithmetic in the operation order the paper prescribes
 *          (Sec. 2.2: density summed then +1 last, alternating-sign velocity
 *          sums, the three-FMA shifted equilibrium of the Sec. 2.2 footnote),
 *          populations quantised through the selected storage codec;
 *   ORD64  the same ordered arithmetic in FP64 (FP64 or FP32 storage).
 *
 * All host arrays are owned by the caller.  Indices are n = x + nx*(y + ny*z)
 * and populations are laid out population-major: f[i*N + n].
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* storage formats (same numbering as the product library's public header,
 * declared independently here) */
enum {
    ORC_FP64 = 0, ORC_FP32 = 1, ORC_FP16 = 2, ORC_FP16S = 3, ORC_FP16C = 4,
    ORC_P16_0S = 5, ORC_P16_1S = 6, ORC_P16_2C = 7, ORC_P16_0 = 8, ORC_P16_1 = 9
};
enum { ORC_D2Q9 = 0, ORC_D3Q19 = 1, ORC_D3Q27 = 2 };
enum { ORC_SRT = 0, ORC_TRT = 1, ORC_MRT = 2 };   /* MRT: D3Q19 only */
enum { ORC_ARITH_DEF64 = 0, ORC_ARITH_ORD32 = 1, ORC_ARITH_ORD64 = 2 };

/* cell flag bits */
#define ORC_WALL      0x01u  /* solid, half-way bounce-back */
#define ORC_MOVING    0x02u  /* with WALL: moving wall, velocity from node_u */
#define ORC_EQ        0x04u  /* equilibrium node (node_rho, node_u) */
#define ORC_OUTFLOW   0x08u  /* zero-gradient outflow in -x direction */
#define ORC_FREESLIP  0x10u  /* with WALL: specular wall, normal axis in bits 5-6 */

/* ---- codecs ---------------------------------------------------------- */
/* 16-bit formats only (FP16..P16_1).  encode: float -> code, decode: code ->
 * float (every code decodes to an exactly representable float). */
uint16_t orc_encode(int fmt, float x);
float    orc_decode(int fmt, uint16_t code);
void orc_encode_array(int fmt, const float* x, uint16_t* out, int64_t n);
void orc_decode_array(int fmt, const uint16_t* c, float* out, int64_t n);
/* encode the floats whose bit patterns are first, first+1, ..., first+n-1 */
void orc_encode_bits_range(int fmt, uint32_t first, int64_t n, uint16_t* out);

/* ---- lattice --------------------------------------------------------- */
typedef struct {
    int nx, ny, nz;
    int velset;        /* ORC_D2Q9 (nz must be 1; every z component of velocity,
                          force and node velocity is ignored), ORC_D3Q19, ORC_D3Q27 */
    int collision;     /* ORC_SRT, ORC_TRT, ORC_MRT (D3Q19) */
    int arith;         /* ORC_ARITH_* */
    int storage;       /* ORC_FP64 for DEF64; any for ORD32; FP64/FP32 for ORD64 */
    double tau;        /* relaxation time, omega = 1/tau */
    double trt_lambda; /* TRT magic parameter (only for ORC_TRT) */
    double force[3];   /* Guo body force per volume, lattice units */
    int no_shift;      /* 0: populations stored shifted, f - w (Sec. 2.2);
                          1: stored as f (appendix, LBM "without DDF-shifting") */
} orc_params;

typedef struct orc_lattice orc_lattice;

int  orc_velset_q(int velset);
/* velocity set tables in the shared direction convention */
void orc_velset_table(int velset, int* c /* q*3 */, double* w /* q */);

orc_lattice* orc_create(const orc_params* p);   /* NULL on bad parameters */
void orc_destroy(orc_lattice* L);
/* flags (N bytes), node_u (3*N floats, component-major: ux[N], uy[N], uz[N]) and
 * node_rho (N floats) may be NULL (all fluid / zero velocity / unit density);
 * the populations of solid cells are set to zero */
/* returns 1 (and changes nothing) if an OUTFLOW cell's -x neighbour is solid */
int orc_set_geometry(orc_lattice* L, const uint8_t* flags, const float* node_u,
                      const float* node_rho);
/* initialise every non-solid cell with the shifted equilibrium of (rho, u) */
void orc_set_rho_u(orc_lattice* L, const double* rho, const double* ux,
                   const double* uy, const double* uz);
/* overwrite the stored populations (q*N, shifted), quantised to the storage
 * format; solid cells are set to zero (their memory is always zero) */
void orc_set_f(orc_lattice* L, const double* f);
void orc_step(orc_lattice* L, int64_t nsteps);
/* density and velocity (incl. the Guo half-force) from the streamed populations */
void orc_get_rho_u(const orc_lattice* L, double* rho, double* ux, double* uy, double* uz);
/* streamed (pulled) populations, shifted, as the next collision sees them;
 * solid cells get 0 */
void orc_get_f(const orc_lattice* L, double* f);
/* FP64 sums over non-solid cells of rho and rho*|u|^2/2 */
void orc_reduce(const orc_lattice* L, double* mass, double* kinetic_energy);
/* D3Q19 MRT moment basis (19 x 19, row-major, in the shared direction
 * order) and the relaxation rate of every moment for relaxation time tau */
void orc_mrt_basis(double* M);
void orc_mrt_rates(double tau, double* s);
/* shifted equilibrium of one cell in the given arithmetic mode (q values) */
void orc_equilibrium(int velset, int arith, double rho, double ux, double uy, double uz, double* feq);
int  orc_threads(void);
/* threads of the following oracle calls (timing only; results do not depend on it) */
void orc_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
