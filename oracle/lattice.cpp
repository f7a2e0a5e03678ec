/*
 * CPU ORACLE -- TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline).
 *
 * Lattice Boltzmann stream-collide of arXiv 2112.08926 as a plain A-B pull
 * loop over cells.  Each step, for every non-solid cell x:
 *   1. streaming (appendix Eq. "lbm-streaming"): f_i(x) = f_i^A(x - e_i), with
 *      half-way bounce-back where x - e_i is solid (Sec. 4.1, mid-grid
 *      bounce-back): f_i(x) = f_ibar^A(x), plus 6 w_i rho_w (c_i . u_w) for a
 *      moving wall (Sec. 4.4 lid, Ladd's rule, rho_w = 1);
 *   2. density with shifted populations (Eq. "rho-shifted"): rho = (sum f_i) + 1
 *      and velocity u = (sum c_i f_i + F/2) / rho (Guo forcing, Sec. 4.1),
 *      each component clamped to +-1/sqrt(3);
 *   3. shifted equilibrium (Eq. "lbm-equilibrium-shifted")
 *      f_i^eq-s = w_i rho (4.5 (u.c_i)^2 - 1.5 u.u + 3 u.c_i) + w_i (rho - 1);
 *   4. collision: SRT (Eq. "lbm-collision") f* = f - (f - f^eq)/tau + (1 - 1/(2 tau)) S_i,
 *      or TRT on the symmetric / antisymmetric parts; Guo source
 *      S_i = w_i (3 (c_i - u) + 9 (c_i . u) c_i) . F;
 *   5. store f* into B at x; then A and B swap.
 * Equilibrium cells store f^eq-s(node_rho, node_u) every step.  Outflow cells
 * take the populations their -x neighbour streams in (zero gradient).  A
 * population streaming out of a free-slip wall is the mirror image (normal
 * component reversed) of the population that hit the wall.
 *
 * Arithmetic modes: DEF64 writes the formulas above directly in FP64.  ORD32
 * and ORD64 follow the operation order the paper prescribes in Sec. 2.2:
 * density summed in index order and 1 added last; velocity sums in
 * alternating + / - order over opposite pairs; each velocity component
 * the momentum component divided by rho (Sec. 2.2, u_x = (f1 - f2 + ...)/rho,
 * and the fields routine of the paper's core, which divides ux, uy and uz by
 * rho one at a time); the shifted equilibrium as
 * A*(0.5*(B^2 + C) +- B) + D with three fused multiply-adds (A = w rho,
 * B = 3 u.c_i, C = -3 u.u, D = w (rho - 1)); SRT as
 * fma(1 - omega, f, omega * f^eq).  Every other operation order used by
 * ORD32/ORD64 is written out in the functions below; this file is compiled
 * with floating-point contraction disabled, so nothing else is fused.
 */
#include "oracle.h"

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

struct VelSet {
    int q = 0, d = 0;
    int c[27][3] = {};
    double w[27] = {};
};

/* Direction convention: 0 is rest; 2k-1 and 2k are opposite; D3Q19 in the
 * order of the paper's D3Q19 core; D3Q27 appends the eight corners. */
VelSet make_velset(int id) {
    VelSet v;
    static const int d3[27][3] = {
        {0, 0, 0},
        {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
        {1, 1, 0}, {-1, -1, 0}, {1, 0, 1}, {-1, 0, -1}, {0, 1, 1}, {0, -1, -1},
        {1, -1, 0}, {-1, 1, 0}, {1, 0, -1}, {-1, 0, 1}, {0, 1, -1}, {0, -1, 1},
        {1, 1, 1}, {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
        {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};
    static const int d2[9][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                                 {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
    if (id == ORC_D2Q9) {
        v.q = 9; v.d = 2;
        std::memcpy(v.c, d2, sizeof d2);
        for (int i = 0; i < 9; ++i) v.w[i] = i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    } else if (id == ORC_D3Q19) {
        v.q = 19; v.d = 3;
        std::memcpy(v.c, d3, 19 * 3 * sizeof(int));
        for (int i = 0; i < 19; ++i) v.w[i] = i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    } else {
        v.q = 27; v.d = 3;
        std::memcpy(v.c, d3, sizeof d3);
        for (int i = 0; i < 27; ++i)
            v.w[i] = i == 0 ? 8.0 / 27.0 : (i < 7 ? 2.0 / 27.0 : (i < 19 ? 1.0 / 54.0 : 1.0 / 216.0));
    }
    return v;
}

inline int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

inline int wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

/* D3Q19 multiple-relaxation-time basis of d'Humieres et al. (2002), the MRT
 * operator the paper's roofline (Sec. 5) lists next to SRT and TRT without
 * defining it.  Rows (moments of the populations): rho, e, epsilon, j_x,
 * q_x, j_y, q_y, j_z, q_z, 3 p_xx, 3 pi_xx, p_ww, pi_ww, p_xy, p_yz, p_xz,
 * m_x, m_y, m_z, as polynomials of the lattice velocity c (|c|^2 = c.c). */
double mrt_entry(int k, const int* c) {
    const double x = c[0], y = c[1], z = c[2], c2 = x * x + y * y + z * z;
    switch (k) {
    case 0: return 1.0;
    case 1: return 19.0 * c2 - 30.0;
    case 2: return (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0;
    case 3: return x;
    case 4: return (5.0 * c2 - 9.0) * x;
    case 5: return y;
    case 6: return (5.0 * c2 - 9.0) * y;
    case 7: return z;
    case 8: return (5.0 * c2 - 9.0) * z;
    case 9: return 3.0 * x * x - c2;
    case 10: return (3.0 * c2 - 5.0) * (3.0 * x * x - c2);
    case 11: return y * y - z * z;
    case 12: return (3.0 * c2 - 5.0) * (y * y - z * z);
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return x * (y * y - z * z);
    case 17: return y * (z * z - x * x);
    default: return z * (x * x - y * y);
    }
}
/* relaxation rates of d'Humieres et al. (2002): the shear moments relax with
 * omega = 1/tau (they set the viscosity), the conserved ones too (their
 * non-equilibrium part is the Guo half force only), the others with fixed
 * rates */
void mrt_rates(double tau, double* s) {
    const double om = 1.0 / tau;
    const double fixed[19] = {om, 1.19, 1.4, om, 1.2, om, 1.2, om, 1.2, om, 1.4, om, 1.4, om, om, om, 1.98, 1.98, 1.98};
    for (int k = 0; k < 19; ++k) s[k] = fixed[k];
}

inline double fmaR(double a, double b, double c) { return std::fma(a, b, c); }
inline float fmaR(float a, float b, float c) { return std::fmaf(a, b, c); }

}  // namespace

struct orc_lattice {
    orc_params p{};
    VelSet vs;
    int64_t N = 0;
    std::vector<uint8_t> flags;
    std::vector<float> nu;    /* 3*N */
    std::vector<float> nrho;  /* N */
    std::vector<double> fa, fb;

    int64_t idx(int x, int y, int z) const { return x + (int64_t)p.nx * (y + (int64_t)p.ny * z); }
    bool solid(int64_t n) const { return flags[n] & ORC_WALL; }
    bool has_force() const { return p.force[0] != 0.0 || p.force[1] != 0.0 || p.force[2] != 0.0; }
};

namespace {

/* value a population takes in memory after a store */
double quantize(const orc_lattice* L, double v) {
    switch (L->p.arith) {
    case ORC_ARITH_DEF64:
        return v;
    case ORC_ARITH_ORD64:
        return L->p.storage == ORC_FP32 ? (double)(float)v : v;
    default: /* ORD32: v is an FP32 value */
        if (L->p.storage == ORC_FP64 || L->p.storage == ORC_FP32) return v;
        return (double)orc_decode(L->p.storage, orc_encode(L->p.storage, (float)v));
    }
}

/* ------------------------------------------------------------------------ */
/* Ordered arithmetic (ORD32 with R = float, ORD64 with R = double).         */
/* ------------------------------------------------------------------------ */
template <class R>
struct Ordered {
    const orc_lattice* L;
    const VelSet& vs;
    R w[27], k6[27], w3[27];
    R om, c1, omp, omm, cSp, cSm, cs, F[3];
    R omph, ommh, cSph, cSmh;   // the TRT rates and source factors halved (exact)
    R sh;   /* 1: shifted populations, 0: unshifted */
    bool force;

    explicit Ordered(const orc_lattice* lat) : L(lat), vs(lat->vs) {
        for (int i = 0; i < vs.q; ++i) {
            w[i] = (R)vs.w[i];
            k6[i] = (R)(6.0 * vs.w[i]);
            w3[i] = (R)(3.0 * vs.w[i]);
        }
        om = (R)(1.0 / L->p.tau);
        c1 = (R)1 - om;
        omp = om;
        const double lam = L->p.trt_lambda;
        omm = (R)(1.0 / (lam / (L->p.tau - 0.5) + 0.5));
        cSp = (R)1 - (R)0.5 * omp;
        cSm = (R)1 - (R)0.5 * omm;
        omph = (R)0.5 * omp;
        ommh = (R)0.5 * omm;
        cSph = (R)0.5 * cSp;
        cSmh = (R)0.5 * cSm;
        cs = (R)(1.0 / std::sqrt(3.0));
        for (int a = 0; a < 3; ++a) F[a] = (R)L->p.force[a];
        force = L->has_force();
        sh = L->p.no_shift ? (R)0 : (R)1;
        if (L->p.collision == ORC_MRT) {
            double s[19];
            mrt_rates(L->p.tau, s);
            for (int k = 0; k < 19; ++k) {
                double norm = 0.0;
                for (int i = 0; i < 19; ++i) {
                    Mk[k][i] = mrt_entry(k, vs.c[i]);
                    norm += Mk[k][i] * Mk[k][i];
                }
                rk[k] = (R)(s[k] / norm);
                pk[k] = (R)((1.0 - 0.5 * s[k]) / norm);
            }
        }
    }
    double Mk[19][19] = {};
    R rk[19] = {}, pk[19] = {};

    /* MRT in a fixed order: d = f - f^eq; m_k = sum_i M_ki d_i (fused
     * multiply-adds over the non-zero M_ki in index order, from +0);
     * n_k = m_k s_k / |M_k|^2; f_i - sum_k M_ki n_k (same order); with
     * forcing, + sum_k M_ki t_k, t_k = (sum_i M_ki S_i)(1 - s_k / 2) / |M_k|^2.
     * M is orthogonal, so sum_k M_ki x_k / |M_k|^2 is M^-1 x. */
    void collide_mrt(R* f, const R* feq, const R* S) const {
        R d[19], n[19], t[19] = {};
        for (int i = 0; i < 19; ++i) d[i] = f[i] - feq[i];
        for (int k = 0; k < 19; ++k) {
            R m = 0, sm = 0;
            for (int i = 0; i < 19; ++i)
                if (Mk[k][i] != 0.0) {
                    m = fmaR((R)Mk[k][i], d[i], m);
                    if (force) sm = fmaR((R)Mk[k][i], S[i], sm);
                }
            n[k] = m * rk[k];
            if (force) t[k] = sm * pk[k];
        }
        for (int i = 0; i < 19; ++i) {
            R acc = 0, acc2 = 0;
            for (int k = 0; k < 19; ++k)
                if (Mk[k][i] != 0.0) {
                    acc = fmaR((R)Mk[k][i], n[k], acc);
                    if (force) acc2 = fmaR((R)Mk[k][i], t[k], acc2);
                }
            f[i] = force ? (f[i] - acc) + acc2 : f[i] - acc;
        }
    }

    /* sum_a c_a * v_a over the non-zero components, in axis order:
     * the first term is +-v_a, each later one is added or subtracted */
    R csum(const int* c, const R* v) const {
        R s = 0;
        bool first = true;
        for (int a = 0; a < 3; ++a) {
            if (c[a] == 0) continue;
            if (first) { s = c[a] > 0 ? v[a] : -v[a]; first = false; }
            else s = c[a] > 0 ? s + v[a] : s - v[a];
        }
        return s;
    }

    R moving_correction(int i, int64_t m) const {
        const int64_t N = L->N;
        const R uw[3] = {(R)L->nu[m], (R)L->nu[N + m], (R)L->nu[2 * N + m]};
        return k6[i] * csum(vs.c[i], uw);
    }

    /* rho (sum in index order, +1 last; +0 for unshifted populations, the
     * appendix's rho = sum f) and the alternating-sign momentum */
    void moments(const R* f, R& rho, R j[3]) const {
        rho = f[0];
        for (int i = 1; i < vs.q; ++i) rho = rho + f[i];
        rho = rho + sh;
        for (int a = 0; a < 3; ++a) {
            R s = 0;
            bool first = true;
            for (int p = 1; p < vs.q; p += 2) {
                const int ca = vs.c[p][a];
                if (ca == 0) continue;
                const int pos = ca > 0 ? p : p + 1, neg = ca > 0 ? p + 1 : p;
                if (first) { s = f[pos] - f[neg]; first = false; }
                else s = (s + f[pos]) - f[neg];
            }
            j[a] = s;
        }
    }

    /* velocity incl. the Guo half-force, before clamping: each momentum
     * component (plus F_a/2, one fused multiply-add) divided by rho, one IEEE
     * division per component, as Sec. 2.2 writes u_x = (f1 - f2 + ...)/rho */
    void velocity(R rho, const R j[3], R u[3]) const {
        for (int a = 0; a < 3; ++a) u[a] = (force ? fmaR((R)0.5, F[a], j[a]) : j[a]) / rho;
    }

    /* three-FMA shifted equilibrium; returns B_p of every pair in Bp.  For
     * unshifted populations D = w rho (rho - 0): the same three FMAs then give
     * w rho (1 + B + (B^2 + C) / 2), the appendix's plain equilibrium. */
    void equilibrium(R rho, const R u[3], R* feq, R* Bp) const {
        R t = u[0] * u[0];
        t = t + u[1] * u[1];
        if (vs.d == 3) t = t + u[2] * u[2];
        const R C = (R)(-3) * t;
        const R u3[3] = {(R)3 * u[0], (R)3 * u[1], (R)3 * u[2]};
        const R rhom1 = rho - sh;
        feq[0] = fmaR(w[0] * rho, (R)0.5 * C, w[0] * rhom1);
        for (int p = 1; p < vs.q; p += 2) {
            const R A = w[p] * rho, D = w[p] * rhom1;
            const R B = csum(vs.c[p], u3);
            const R X = fmaR(B, B, C);
            feq[p] = fmaR(A, fmaR((R)0.5, X, B), D);
            feq[p + 1] = fmaR(A, fmaR((R)0.5, X, -B), D);
            Bp[p] = B;
        }
    }

    /* Guo source S_i = 3 w_i ((c_i.F - u.F) + B_i (c_i.F)), B_i = 3 c_i.u */
    void source(const R u[3], const R* Bp, R* S) const {
        R uF = u[0] * F[0];
        uF = fmaR(u[1], F[1], uF);
        if (vs.d == 3) uF = fmaR(u[2], F[2], uF);
        S[0] = w3[0] * (-uF);
        for (int p = 1; p < vs.q; p += 2) {
            const R cF = csum(vs.c[p], F);
            const R B = Bp[p];
            S[p] = w3[p] * fmaR(B, cF, cF - uF);
            S[p + 1] = w3[p] * fmaR(B, cF, (-cF) - uF);
        }
    }

    /* f: streamed populations -> post-collision populations, in place */
    void collide(R* f) const {
        R rho, j[3], u[3];
        moments(f, rho, j);
        velocity(rho, j, u);
        for (int a = 0; a < 3; ++a) u[a] = std::fmin(std::fmax(u[a], -cs), cs);
        R feq[27], Bp[27] = {}, S[27] = {};
        equilibrium(rho, u, feq, Bp);
        if (force) source(u, Bp, S);
        if (L->p.collision == ORC_MRT) {
            collide_mrt(f, feq, S);
        } else if (L->p.collision == ORC_SRT) {
            for (int i = 0; i < vs.q; ++i)
                f[i] = force ? fmaR(c1, f[i], fmaR(om, feq[i], cSp * S[i]))
                             : fmaR(c1, f[i], om * feq[i]);
        } else {
            const R a0 = f[0] - feq[0];
            f[0] = fmaR(-omp, a0, force ? fmaR(cSp, S[0], f[0]) : f[0]);
            for (int p = 1; p < vs.q; p += 2) {
                const int q = p + 1;
                // symmetric and antisymmetric parts of the pair, (a + b)/2 and
                // (a - b)/2, relaxed with omega+ and omega-; the halves ride
                // on the rates: omega/2 (a + b) is one product, exact halving
                const R a = f[p] - feq[p], b = f[q] - feq[q];
                const R s = a + b, d = a - b;
                R fp = f[p], fq = f[q];
                if (force) {   // (1 - omega+/2) and (1 - omega-/2) on the source's parts
                    const R Ss = S[p] + S[q], Sd = S[p] - S[q];
                    fp = fp + fmaR(cSmh, Sd, cSph * Ss);
                    fq = fq + fmaR(-cSmh, Sd, cSph * Ss);
                }
                f[p] = fmaR(-ommh, d, fmaR(-omph, s, fp));
                f[q] = fmaR(ommh, d, fmaR(-omph, s, fq));
            }
        }
    }

    void equilibrium_only(R rho, const R u[3], R* feq) const {
        R Bp[27];
        equilibrium(rho, u, feq, Bp);
    }

    void fields(const R* f, R& rho, R u[3]) const {
        R j[3];
        moments(f, rho, j);
        velocity(rho, j, u);
    }
};

/* inverse of a 19 x 19 matrix by Gauss-Jordan elimination with partial pivoting */
void invert19(const double (*A)[19], double (*X)[19]) {
    double a[19][38];
    for (int r = 0; r < 19; ++r)
        for (int c = 0; c < 38; ++c) a[r][c] = c < 19 ? A[r][c] : (c - 19 == r ? 1.0 : 0.0);
    for (int col = 0; col < 19; ++col) {
        int piv = col;
        for (int r = col + 1; r < 19; ++r)
            if (std::fabs(a[r][col]) > std::fabs(a[piv][col])) piv = r;
        for (int c = 0; c < 38; ++c) std::swap(a[col][c], a[piv][c]);
        const double d = a[col][col];
        for (int c = 0; c < 38; ++c) a[col][c] /= d;
        for (int r = 0; r < 19; ++r)
            if (r != col) {
                const double m = a[r][col];
                if (m != 0.0)
                    for (int c = 0; c < 38; ++c) a[r][c] -= m * a[col][c];
            }
    }
    for (int r = 0; r < 19; ++r)
        for (int c = 0; c < 19; ++c) X[r][c] = a[r][19 + c];
}

/* ------------------------------------------------------------------------ */
/* Definition in FP64 (DEF64).                                               */
/* ------------------------------------------------------------------------ */
struct Definition {
    const orc_lattice* L;
    const VelSet& vs;
    explicit Definition(const orc_lattice* lat) : L(lat), vs(lat->vs) {}

    double dot(const int* c, const double* v) const { return c[0] * v[0] + c[1] * v[1] + c[2] * v[2]; }

    double moving_correction(int i, int64_t m) const {
        const int64_t N = L->N;
        const double uw[3] = {L->nu[m], L->nu[N + m], L->nu[2 * N + m]};
        return 6.0 * vs.w[i] * 1.0 * dot(vs.c[i], uw);   /* rho_w = 1 */
    }

    void fields(const double* f, double& rho, double u[3]) const {
        double s = 0, j[3] = {0, 0, 0};
        for (int i = 0; i < vs.q; ++i) {
            s += f[i];
            for (int a = 0; a < 3; ++a) j[a] += vs.c[i][a] * f[i];
        }
        rho = L->p.no_shift ? s : s + 1.0;   /* Sec. 2.2 / appendix without shifting */
        for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * L->p.force[a]) / rho;
    }

    void equilibrium_only(double rho, const double u[3], double* feq) const {
        const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        for (int i = 0; i < vs.q; ++i) {
            const double cu = dot(vs.c[i], u);
            if (L->p.no_shift)   /* appendix, equilibrium without DDF-shifting */
                feq[i] = vs.w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
            else                 /* Sec. 2.2, shifted equilibrium */
                feq[i] = vs.w[i] * rho * (4.5 * cu * cu - 1.5 * uu + 3.0 * cu) + vs.w[i] * (rho - 1.0);
        }
    }

    void collide(double* f) const {
        double rho, u[3];
        fields(f, rho, u);
        const double cs = 1.0 / std::sqrt(3.0);
        for (int a = 0; a < 3; ++a) u[a] = std::fmin(std::fmax(u[a], -cs), cs);
        double feq[27], S[27];
        equilibrium_only(rho, u, feq);
        const double* F = L->p.force;
        const double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
        for (int i = 0; i < vs.q; ++i) {
            const double cu = dot(vs.c[i], u), cF = dot(vs.c[i], F);
            S[i] = vs.w[i] * (3.0 * (cF - uF) + 9.0 * cu * cF);
        }
        const double omega = 1.0 / L->p.tau;
        if (L->p.collision == ORC_MRT) {
            /* f* = f - M^-1 S_diag M (f - f^eq) + M^-1 (I - S_diag / 2) M S_guo */
            double M[19][19], Minv[19][19], s[19], m[19], g[19];
            for (int k = 0; k < 19; ++k)
                for (int i = 0; i < 19; ++i) M[k][i] = mrt_entry(k, vs.c[i]);
            invert19(M, Minv);
            mrt_rates(L->p.tau, s);
            for (int k = 0; k < 19; ++k) {
                double neq = 0.0, src = 0.0;
                for (int i = 0; i < 19; ++i) {
                    neq += M[k][i] * (f[i] - feq[i]);
                    src += M[k][i] * S[i];
                }
                m[k] = -s[k] * neq + (1.0 - 0.5 * s[k]) * src;
            }
            for (int i = 0; i < 19; ++i) {
                g[i] = f[i];
                for (int k = 0; k < 19; ++k) g[i] += Minv[i][k] * m[k];
            }
            for (int i = 0; i < 19; ++i) f[i] = g[i];
        } else if (L->p.collision == ORC_SRT) {
            for (int i = 0; i < vs.q; ++i)
                f[i] = f[i] - omega * (f[i] - feq[i]) + (1.0 - 0.5 * omega) * S[i];
        } else {
            const double omm = 1.0 / (L->p.trt_lambda / (L->p.tau - 0.5) + 0.5);
            double g[27];
            for (int i = 0; i < vs.q; ++i) {
                const int b = opp(i);
                const double fp = 0.5 * (f[i] + f[b]), fm = 0.5 * (f[i] - f[b]);
                const double ep = 0.5 * (feq[i] + feq[b]), em = 0.5 * (feq[i] - feq[b]);
                const double Sp = 0.5 * (S[i] + S[b]), Sm = 0.5 * (S[i] - S[b]);
                g[i] = f[i] - omega * (fp - ep) - omm * (fm - em) + (1.0 - 0.5 * omega) * Sp +
                       (1.0 - 0.5 * omm) * Sm;
            }
            for (int i = 0; i < vs.q; ++i) f[i] = g[i];
        }
    }
};

/* streamed population i for a cell that sits (for streaming) at (sx,sy,sz) */
template <class R, class Ar>
R pull(const orc_lattice* L, const Ar& ar, int sx, int sy, int sz, int i) {
    const VelSet& vs = L->vs;
    const int64_t N = L->N;
    const int* c = vs.c[i];
    const int yx = wrap(sx - c[0], L->p.nx), yy = wrap(sy - c[1], L->p.ny), yz = wrap(sz - c[2], L->p.nz);
    const int64_t m = L->idx(yx, yy, yz);
    const uint8_t fy = L->flags[m];
    if (!(fy & ORC_WALL)) return (R)L->fa[i * N + m];
    if (fy & ORC_FREESLIP) {
        const int axis = (fy >> 5) & 3;
        if (axis < 3) {
            int mc[3] = {c[0], c[1], c[2]};
            mc[axis] = -mc[axis];
            int mi = 0;
            while (mi < vs.q && !(vs.c[mi][0] == mc[0] && vs.c[mi][1] == mc[1] && vs.c[mi][2] == mc[2])) ++mi;
            int t[3] = {yx, yy, yz};
            const int s[3] = {sx, sy, sz};
            t[axis] = s[axis];
            const int64_t m2 = L->idx(t[0], t[1], t[2]);
            if (!(L->flags[m2] & ORC_WALL)) return (R)L->fa[mi * N + m2];
        }
    }
    R v = (R)L->fa[opp(i) * N + L->idx(sx, sy, sz)];
    if (fy & ORC_MOVING) v = v + ar.moving_correction(i, m);
    return v;
}

template <class R, class Ar>
void pull_cell(const orc_lattice* L, const Ar& ar, int x, int y, int z, R* f) {
    int sx = x;
    if (L->flags[L->idx(x, y, z)] & ORC_OUTFLOW) sx = wrap(x - 1, L->p.nx);
    for (int i = 0; i < L->vs.q; ++i) f[i] = pull<R>(L, ar, sx, y, z, i);
}

template <class R, class Ar>
void step_once(orc_lattice* L, const Ar& ar) {
    const int64_t N = L->N;
    const int q = L->vs.q;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < L->p.nz; ++z) {
        for (int y = 0; y < L->p.ny; ++y) {
            for (int x = 0; x < L->p.nx; ++x) {
                const int64_t n = L->idx(x, y, z);
                const uint8_t fl = L->flags[n];
                R f[27];
                if (fl & ORC_WALL) continue;
                if (fl & ORC_EQ) {
                    const R u[3] = {(R)L->nu[n], (R)L->nu[N + n], (R)L->nu[2 * N + n]};
                    ar.equilibrium_only((R)L->nrho[n], u, f);
                } else {
                    pull_cell<R>(L, ar, x, y, z, f);
                    ar.collide(f);
                }
                for (int i = 0; i < q; ++i) L->fb[i * N + n] = quantize(L, (double)f[i]);
            }
        }
    }
    L->fa.swap(L->fb);
}

template <class R, class Ar>
void get_fields(const orc_lattice* L, const Ar& ar, double* rho, double* ux, double* uy, double* uz) {
    const int64_t N = L->N;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < L->p.nz; ++z)
        for (int y = 0; y < L->p.ny; ++y)
            for (int x = 0; x < L->p.nx; ++x) {
                const int64_t n = L->idx(x, y, z);
                const uint8_t fl = L->flags[n];
                double r = 1.0, u[3] = {0, 0, 0};
                if (fl & ORC_WALL) {
                } else if (fl & ORC_EQ) {
                    r = L->nrho[n];
                    for (int a = 0; a < 3; ++a) u[a] = L->nu[a * N + n];
                } else {
                    R f[27], rr, uu[3];
                    pull_cell<R>(L, ar, x, y, z, f);
                    ar.fields(f, rr, uu);
                    r = (double)rr;
                    for (int a = 0; a < 3; ++a) u[a] = (double)uu[a];
                }
                if (rho) rho[n] = r;
                if (ux) ux[n] = u[0];
                if (uy) uy[n] = u[1];
                if (uz) uz[n] = u[2];
            }
}

template <class R, class Ar>
void get_pulled(const orc_lattice* L, const Ar& ar, double* out) {
    const int64_t N = L->N;
    const int q = L->vs.q;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < L->p.nz; ++z)
        for (int y = 0; y < L->p.ny; ++y)
            for (int x = 0; x < L->p.nx; ++x) {
                const int64_t n = L->idx(x, y, z);
                R f[27];
                if (L->flags[n] & ORC_WALL) {
                    for (int i = 0; i < q; ++i) out[i * N + n] = 0.0;
                    continue;
                }
                pull_cell<R>(L, ar, x, y, z, f);
                for (int i = 0; i < q; ++i) out[i * N + n] = (double)f[i];
            }
}

template <class R, class Ar>
void init_eq(orc_lattice* L, const Ar& ar, const double* rho, const double* ux, const double* uy,
             const double* uz) {
    const int64_t N = L->N;
    const int q = L->vs.q;
    for (int64_t n = 0; n < N; ++n) {
        if (L->solid(n)) {
            for (int i = 0; i < q; ++i) L->fa[i * N + n] = 0.0;
            continue;
        }
        const R u[3] = {(R)(ux ? ux[n] : 0.0), (R)(uy ? uy[n] : 0.0),
                        (R)(uz && L->vs.d == 3 ? uz[n] : 0.0)};
        R feq[27];
        ar.equilibrium_only((R)(rho ? rho[n] : 1.0), u, feq);
        for (int i = 0; i < q; ++i) L->fa[i * N + n] = quantize(L, (double)feq[i]);
    }
}

template <class Fn>
void dispatch(const orc_lattice* L, Fn fn) {
    if (L->p.arith == ORC_ARITH_DEF64) fn(Definition(L), (double*)nullptr);
    else if (L->p.arith == ORC_ARITH_ORD64) fn(Ordered<double>(L), (double*)nullptr);
    else fn(Ordered<float>(L), (float*)nullptr);
}

}  // namespace

extern "C" {

int orc_velset_q(int velset) {
    return velset == ORC_D2Q9 ? 9 : velset == ORC_D3Q19 ? 19 : velset == ORC_D3Q27 ? 27 : 0;
}

void orc_velset_table(int velset, int* c, double* w) {
    const VelSet v = make_velset(velset);
    for (int i = 0; i < v.q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = v.c[i][a];
        w[i] = v.w[i];
    }
}

orc_lattice* orc_create(const orc_params* p) {
    if (!p || p->nx < 1 || p->ny < 1 || p->nz < 1) return nullptr;
    if (orc_velset_q(p->velset) == 0) return nullptr;
    if (p->velset == ORC_D2Q9 && p->nz != 1) return nullptr;
    if (p->collision != ORC_SRT && p->collision != ORC_TRT && p->collision != ORC_MRT) return nullptr;
    if (p->collision == ORC_MRT && p->velset != ORC_D3Q19) return nullptr;
    if (!(p->tau > 0.5)) return nullptr;
    if (p->arith == ORC_ARITH_DEF64 && p->storage != ORC_FP64) return nullptr;
    if (p->arith == ORC_ARITH_ORD64 && p->storage != ORC_FP64 && p->storage != ORC_FP32) return nullptr;
    if (p->storage < ORC_FP64 || p->storage > ORC_P16_1) return nullptr;
    orc_lattice* L = new orc_lattice;
    L->p = *p;
    if (p->velset == ORC_D2Q9) L->p.force[2] = 0.0;   /* D2Q9 ignores every z component */
    L->vs = make_velset(p->velset);
    L->N = (int64_t)p->nx * p->ny * p->nz;
    L->flags.assign(L->N, 0);
    L->nu.assign(3 * L->N, 0.0f);
    L->nrho.assign(L->N, 1.0f);
    L->fa.assign(L->vs.q * L->N, 0.0);
    L->fb.assign(L->vs.q * L->N, 0.0);
    if (p->no_shift) orc_set_rho_u(L, nullptr, nullptr, nullptr, nullptr);   /* rest is not zero */
    return L;
}

void orc_destroy(orc_lattice* L) { delete L; }

int orc_set_geometry(orc_lattice* L, const uint8_t* flags, const float* node_u, const float* node_rho) {
    const int64_t N = L->N;
    /* an outflow cell pulls as if it sat one cell upstream in x; that cell
     * must hold populations */
    if (flags)
        for (int64_t n = 0; n < N; ++n) {
            if (!(flags[n] & ORC_OUTFLOW)) continue;
            const int x = (int)(n % L->p.nx);
            const int64_t m = n - x + (x == 0 ? L->p.nx - 1 : x - 1);
            if (flags[m] & ORC_WALL) return 1;
        }
    if (flags) std::memcpy(L->flags.data(), flags, N);
    else std::fill(L->flags.begin(), L->flags.end(), 0);
    if (node_u) std::memcpy(L->nu.data(), node_u, 3 * N * sizeof(float));
    else std::fill(L->nu.begin(), L->nu.end(), 0.0f);
    if (L->vs.d == 2) std::fill(L->nu.begin() + 2 * N, L->nu.end(), 0.0f);
    if (node_rho) std::memcpy(L->nrho.data(), node_rho, N * sizeof(float));
    else std::fill(L->nrho.begin(), L->nrho.end(), 1.0f);
    /* solid cells hold no populations */
    for (int64_t n = 0; n < N; ++n)
        if (L->solid(n))
            for (int i = 0; i < L->vs.q; ++i) L->fa[i * N + n] = L->fb[i * N + n] = 0.0;
    return 0;
}

void orc_set_rho_u(orc_lattice* L, const double* rho, const double* ux, const double* uy, const double* uz) {
    dispatch(L, [&](const auto& ar, auto* tag) {
        using R = std::remove_pointer_t<decltype(tag)>;
        init_eq<R>(L, ar, rho, ux, uy, uz);
    });
    std::fill(L->fb.begin(), L->fb.end(), 0.0);
}

void orc_set_f(orc_lattice* L, const double* f) {
    const int64_t N = L->N;
    std::fill(L->fb.begin(), L->fb.end(), 0.0);
    for (int i = 0; i < L->vs.q; ++i)
        for (int64_t n = 0; n < N; ++n)
            L->fa[i * N + n] = L->solid(n) ? 0.0 : quantize(L, f[i * N + n]);
}

void orc_step(orc_lattice* L, int64_t nsteps) {
    dispatch(L, [&](const auto& ar, auto* tag) {
        using R = std::remove_pointer_t<decltype(tag)>;
        for (int64_t s = 0; s < nsteps; ++s) step_once<R>(L, ar);
    });
}

void orc_get_rho_u(const orc_lattice* L, double* rho, double* ux, double* uy, double* uz) {
    dispatch(L, [&](const auto& ar, auto* tag) {
        using R = std::remove_pointer_t<decltype(tag)>;
        get_fields<R>(L, ar, rho, ux, uy, uz);
    });
}

void orc_get_f(const orc_lattice* L, double* f) {
    dispatch(L, [&](const auto& ar, auto* tag) {
        using R = std::remove_pointer_t<decltype(tag)>;
        get_pulled<R>(L, ar, f);
    });
}

void orc_equilibrium(int velset, int arith, double rho, double ux, double uy, double uz, double* feq) {
    orc_params p{};
    p.nx = p.ny = p.nz = 1;
    p.velset = velset;
    p.collision = ORC_SRT;
    p.arith = arith;
    p.storage = arith == ORC_ARITH_ORD32 ? ORC_FP32 : ORC_FP64;
    p.tau = 1.0;
    orc_lattice* L = orc_create(&p);
    if (!L) return;
    dispatch(L, [&](const auto& ar, auto* tag) {
        using R = std::remove_pointer_t<decltype(tag)>;
        const R u[3] = {(R)ux, (R)uy, (R)uz};
        R e[27];
        ar.equilibrium_only((R)rho, u, e);
        for (int i = 0; i < L->vs.q; ++i) feq[i] = (double)e[i];
    });
    orc_destroy(L);
}

void orc_reduce(const orc_lattice* L, double* mass, double* kinetic_energy) {
    const int64_t N = L->N;
    std::vector<double> r(N), ux(N), uy(N), uz(N);
    orc_get_rho_u(L, r.data(), ux.data(), uy.data(), uz.data());
    double m = 0.0, e = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        if (L->solid(n)) continue;
        m += r[n];
        e += 0.5 * r[n] * (ux[n] * ux[n] + uy[n] * uy[n] + uz[n] * uz[n]);
    }
    if (mass) *mass = m;
    if (kinetic_energy) *kinetic_energy = e;
}

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

}  // extern "C"

void orc_mrt_basis(double* M) {
    const VelSet vs = make_velset(ORC_D3Q19);
    for (int k = 0; k < 19; ++k)
        for (int i = 0; i < 19; ++i) M[k * 19 + i] = mrt_entry(k, vs.c[i]);
}

void orc_mrt_rates(double tau, double* s) { mrt_rates(tau, s); }
