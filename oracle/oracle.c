/*
 * oracle.c -- plain FP64 CPU oracle for the IMEXLBM per-time-step update.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, table, header or constant with the
 * CUDA library; the two meet only through seeded inputs produced elsewhere.
 *
 * What it computes (arxiv 2201.11330, "IMEXLBM 1.0"):
 *   Sec. 2.1  discrete velocity models (D2Q9 table printed in Sec. 2.1; D3Q19
 *             and D3Q27 after Qian et al. 1992, which Sec. 2.1 cites),
 *             Eq. (feq) compressible equilibrium, Eq. (incompressible_feq)
 *             incompressible equilibrium, Eq. (collision) IMEX/trapezoidal
 *             BGK relaxation with omega = 1/(tau_paper + 1/2), Eq.
 *             (propagation), and the moment definitions p = c_s^2 sum f,
 *             u = (1/rho) sum e f.
 *   Sec. 2.2  initialisation by equilibrium, no-slip bounce-back Eq. (bb).
 *   Sec. 3.1  step order: Collision -> BoundaryCondition -> Propagation ->
 *             PostProcessing.
 *
 * Readings of points the paper leaves open (each one is a decision, listed
 * with its reason in the design notes):
 *   - tau passed here is the standard BGK time tau_std = tau_paper + 1/2, so
 *     omega = 1/tau_std and nu = c_s^2 (tau_std - 1/2).
 *   - incompressible model: u = (sum e f + F/2)/rho0; compressible model:
 *     rho = sum f, u = (sum e f + F/2)/rho.
 *   - D3Q19 / D3Q27 numbering: lexicographic in (e_x, e_y, e_z), e_x slowest,
 *     the same rule the printed D2Q9 table follows.
 *   - bounce-back is the half-way link form applied before propagation: a
 *     population whose upstream node lies beyond a wall is replaced by the
 *     node's own post-collision population of the opposite direction.
 *   - moving wall (not in the paper): Ladd's term 2 t_a rho0 (e_a . U)/c_s^2
 *     on links whose upstream node has y >= ny (the +y face, corners
 *     included).
 *   - body force (not in the paper): Guo forcing in the same trapezoidal
 *     form, source (1 - omega/2) t_a [(e_a - u).F/c_s^2 + (e_a.u)(e_a.F)/c_s^4].
 *   - adjoint (not in the paper): the exact transpose of one step, objective
 *     J = rho0/2 sum_x |u(x, T)|^2.
 *   - two-relaxation-time collision (not in the paper; Ginzburg's TRT): the
 *     pair halves f+ = (f_a + f_abar)/2 and f- = (f_a - f_abar)/2 relax at
 *     omega and omega_m, Lambda = (1/omega - 1/2)(1/omega_m - 1/2); the Guo
 *     source splits the same way, its even half scaled by (1 - omega/2), its
 *     odd half by (1 - omega_m/2).  Lambda = 0 selects BGK.
 *   - multiple-relaxation-time collision (not in the paper; d'Humieres et al.
 *     2002): f*_a = f_a - sum_k M_ka [s_k m_k(f - feq) - (1 - s_k/2) m_k(S)]
 *     / |M_k|^2 with m_k(g) = sum_a M_ka g_a, S the Guo source without its
 *     (1 - omega/2) factor, and M the moment basis orthogonal over the
 *     velocity set: the monomials e_x^i e_y^j e_z^k (i, j, k <= 2) taken by
 *     degree, |e|^2 first among degree two, orthogonalised in that order
 *     (Gram-Schmidt), linearly dependent ones dropped.  Rates by class:
 *     density and momentum (conserved; any rate gives the same result), the
 *     bulk row from |e|^2 at s_bulk, the other second-order rows (the
 *     traceless stress) at omega, higher rows at s_even or s_odd by the
 *     parity of their degree.  All rates = omega gives BGK; s_bulk = s_even
 *     = omega and s_odd = omega_m give TRT.
 *   - per-face boundaries and obstacles (Sec. 4-5 use them; their discrete
 *     form is not printed): for the population entering fluid node x along
 *     e_a, take the upstream node x - e_a and fix each coordinate that
 *     leaves the box by the type of the face it crosses: periodic wraps;
 *     wall and inlet bounce back half-way (f_a(x) = f*_abar(x) plus
 *     2 t_a rho0 (e_a . U)/c_s^2 with U the inlet velocity at x for an
 *     inlet, the lid velocity for the +y wall, else 0; the inlet wins over
 *     the lid on a link crossing both); outflow is a pressure outlet by
 *     anti-bounce-back, f_a(x) = -f*_abar(x) + 2 feq+_a(P_out, u(x)) with
 *     feq+ the even half of the equilibrium and u(x) the node's velocity from
 *     its post-collision populations (the paper's convective outflow is not
 *     printed; a velocity inlet needs a pressure level fixed somewhere, and a
 *     zero-gradient outlet leaves it free to drift); symmetry mirrors the
 *     coordinate back to that of x and reflects the direction's component
 *     normal to the face (specular, free slip); nodal is the paper's own
 *     "modified nodal bounce-back" of Sec. 2.2 (Eq. (bb), Ziegler): the wall
 *     lies on the boundary nodes, which collide like the bulk, and a
 *     population entering one from outside is the one of the opposite
 *     direction that has just arrived there from inside, f_a(x) = f_abar(x)
 *     after propagation (plus the lid term on the +y face; where that
 *     opposite population comes from outside too, as at a corner, the
 *     node's own f*_abar(x) is taken).  Crossings rank wall/inlet, then
 *     nodal, then outflow, then symmetry/periodic.  If the node so found is solid, the
 *     population bounces back at x as well (stationary obstacle), and the
 *     link's momentum exchange 2 f*_abar(x) e_abar counts towards the
 *     force on the obstacle (Sec. 5, momentum exchange of Ladd).  Solid
 *     nodes are not updated; PostProcessing reports p = 0, u = 0 there.
 *
 * Pins (tests under tests/ check these against closed forms, conservation
 * laws, analytic flows and finite differences): tables, equilibrium moments,
 * collision invariants, conservation under streaming, Taylor-Green decay,
 * Poiseuille and Couette profiles, the rest state, the pressure gauge, and
 * the adjoint against central differences of or_run.  No function here is
 * parity-unpinned.
 *
 * Layout: distributions are kept like the paper's arrays, node-major with the
 * direction fastest (f[node*Q + a]).  Arrays crossing the interface are
 * structure-of-arrays (component-major) FP64.  Node index n = x + nx*(y + ny*z).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXQ 27

enum { OR_D2Q9 = 0, OR_D3Q19 = 1, OR_D3Q27 = 2 };
enum { OR_BC_PERIODIC = 0, OR_BC_CAVITY = 1, OR_BC_CHANNEL = 2 };
enum { OR_FACE_PERIODIC = 0, OR_FACE_WALL = 1, OR_FACE_INLET = 2, OR_FACE_OUTFLOW = 3,
       OR_FACE_SYMMETRY = 4, OR_FACE_NODAL = 5 };
enum { OR_LINK_STREAM = 0, OR_LINK_WALL = 1, OR_LINK_SOLID = 2, OR_LINK_OUTFLOW = 3,
       OR_LINK_NODAL = 4 };
enum { OR_OK = 0, OR_ERR_ARG = -1, OR_ERR_NOMEM = -5 };

/* 1/c_s^2 for all three velocity sets (c_s^2 = c^2/3, c = 1). */
static const double INV_CS2 = 3.0;

typedef struct {
    int Q, d;
    int e[OR_MAXQ][3];
    double t[OR_MAXQ];
    int opp[OR_MAXQ];
} or_dvm;

typedef struct {
    or_dvm v;
    int nx, ny, nz;
    long N;
    int periodic[3];
    int lid_on;
    int face[6];                 /* face types, order -x, +x, -y, +y, -z, +z */
    const unsigned char *solid;  /* N, nonzero = solid node, or NULL */
    const double *inlet_u;       /* d * (nodes of the inlet face), or NULL */
    double P_out;                /* outflow pressure level P = p / c_s^2 */
    double lid[3];
    double omega, rho0;
    double omega_m; /* TRT odd-part rate; 0 = BGK */
    int mrt;        /* MRT collision with the basis and rates below */
    int nrow;       /* rows of the moment basis (= Q) */
    double M[OR_MAXQ][OR_MAXQ], M2[OR_MAXQ], s_row[OR_MAXQ];
    int compressible;
    const double *F; /* d*N, component-major, or NULL */
} or_model;

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: discrete velocity models.                                       */

static int build_dvm(int lattice, or_dvm *v)
{
    memset(v, 0, sizeof(*v));
    if (lattice == OR_D2Q9) {
        /* The D2Q9 velocity matrix and weight vector as printed in Sec. 2.1
         * (first row e_x, second row e_y). */
        static const int ex[9] = {-1, -1, -1, 0, 0, 0, 1, 1, 1};
        static const int ey[9] = {-1, 0, 1, -1, 0, 1, -1, 0, 1};
        static const double w[9] = {1.0 / 36, 1.0 / 9, 1.0 / 36, 1.0 / 9, 4.0 / 9,
                                    1.0 / 9,  1.0 / 36, 1.0 / 9, 1.0 / 36};
        v->Q = 9;
        v->d = 2;
        for (int a = 0; a < 9; ++a) {
            v->e[a][0] = ex[a];
            v->e[a][1] = ey[a];
            v->e[a][2] = 0;
            v->t[a] = w[a];
        }
    } else if (lattice == OR_D3Q19 || lattice == OR_D3Q27) {
        /* Qian et al. (1992) weights by speed class |e|^2 = 0, 1, 2, 3. */
        static const double w19[4] = {1.0 / 3, 1.0 / 18, 1.0 / 36, 0.0};
        static const double w27[4] = {8.0 / 27, 2.0 / 27, 1.0 / 54, 1.0 / 216};
        const double *w = (lattice == OR_D3Q19) ? w19 : w27;
        int q = 0;
        for (int x = -1; x <= 1; ++x)
            for (int y = -1; y <= 1; ++y)
                for (int z = -1; z <= 1; ++z) {
                    int s = x * x + y * y + z * z;
                    if (lattice == OR_D3Q19 && s == 3)
                        continue;
                    v->e[q][0] = x;
                    v->e[q][1] = y;
                    v->e[q][2] = z;
                    v->t[q] = w[s];
                    ++q;
                }
        v->Q = q;
        v->d = 3;
    } else {
        return OR_ERR_ARG;
    }
    /* opposite direction found by search, so that the numbering rule of
     * Sec. 2.1 (opposite = Q-1-a) is something the tests can check. */
    for (int a = 0; a < v->Q; ++a) {
        v->opp[a] = -1;
        for (int b = 0; b < v->Q; ++b)
            if (v->e[b][0] == -v->e[a][0] && v->e[b][1] == -v->e[a][1] &&
                v->e[b][2] == -v->e[a][2])
                v->opp[a] = b;
    }
    return OR_OK;
}

/* Exported: the velocity set, for the table pins. e is Q*3 ints. */
int or_tables(int lattice, int *Q, int *d, int *e, double *t, int *opp)
{
    or_dvm v;
    if (build_dvm(lattice, &v) != OR_OK)
        return OR_ERR_ARG;
    *Q = v.Q;
    *d = v.d;
    for (int a = 0; a < v.Q; ++a) {
        for (int k = 0; k < 3; ++k)
            e[3 * a + k] = v.e[a][k];
        t[a] = v.t[a];
        opp[a] = v.opp[a];
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: equilibrium.                                                    */

/* Eq. (incompressible_feq) when compressible == 0:
 *     feq_a = t_a [ P + rho0 ( e.u/c_s^2 + (e.u)^2/(2 c_s^4) - u.u/(2 c_s^2) ) ]
 * with P = p/c_s^2.  Eq. (feq) when compressible == 1:
 *     feq_a = t_a rho [ 1 + e.u/c_s^2 + (e.u)^2/(2 c_s^4) - u.u/(2 c_s^2) ]
 * with rho = P. */
static void equilibrium(const or_dvm *v, int compressible, double rho0, double P,
                        const double u[3], double *feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int a = 0; a < v->Q; ++a) {
        double eu = v->e[a][0] * u[0] + v->e[a][1] * u[1] + v->e[a][2] * u[2];
        double poly = eu * INV_CS2 + 0.5 * eu * eu * INV_CS2 * INV_CS2 - 0.5 * uu * INV_CS2;
        if (compressible)
            feq[a] = v->t[a] * P * (1.0 + poly);
        else
            feq[a] = v->t[a] * (P + rho0 * poly);
    }
}

/* Exported: one node's equilibrium (for the moment pins). */
int or_equilibrium(int lattice, int compressible, double rho0, double P,
                   const double *u3, double *feq)
{
    or_dvm v;
    if (build_dvm(lattice, &v) != OR_OK)
        return OR_ERR_ARG;
    double u[3] = {u3[0], u3[1], u3[2]};
    equilibrium(&v, compressible, rho0, P, u, feq);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: moments p = c_s^2 sum f, u = (1/rho) sum e f (+ F/2, Guo).     */

static void node_moments(const or_model *m, const double *fn, const double *Fn,
                         double *P, double u[3])
{
    const or_dvm *v = &m->v;
    double s = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < v->Q; ++a) {
        s += fn[a];
        for (int k = 0; k < 3; ++k)
            j[k] += v->e[a][k] * fn[a];
    }
    double rho = m->compressible ? s : m->rho0;
    for (int k = 0; k < 3; ++k)
        u[k] = (j[k] + (Fn ? 0.5 * Fn[k] : 0.0)) / rho;
    *P = s;
}

static void load_force(const or_model *m, long n, double Fn[3])
{
    Fn[0] = Fn[1] = Fn[2] = 0.0;
    if (!m->F)
        return;
    for (int k = 0; k < m->v.d; ++k)
        Fn[k] = m->F[(long)k * m->N + n];
}

/* TRT collision (not in the paper): with g+ = (g_a + g_abar)/2 and
 * g- = (g_a - g_abar)/2 for g = f, feq and the Guo source S,
 *     f*_a = f_a - omega (f+ - feq+) - omega_m (f- - feq-)
 *            + (1 - omega/2) S+ + (1 - omega_m/2) S-.
 * Overwrites out[] (the BGK result) with this. */
static void guo_source(const or_dvm *v, int a, const double u[3], const double *Fn, double *S)
{
    *S = 0.0;
    if (!Fn)
        return;
    double eu = v->e[a][0] * u[0] + v->e[a][1] * u[1] + v->e[a][2] * u[2];
    double eF = v->e[a][0] * Fn[0] + v->e[a][1] * Fn[1] + v->e[a][2] * Fn[2];
    double uF = u[0] * Fn[0] + u[1] * Fn[1] + u[2] * Fn[2];
    *S = v->t[a] * ((eF - uF) * INV_CS2 + eu * eF * INV_CS2 * INV_CS2);
}

static void collide_node_trt(const or_model *m, const double *fn, const double *Fn,
                             const double *feq, const double u[3], double *out)
{
    const or_dvm *v = &m->v;
    for (int a = 0; a < v->Q; ++a) {
        int b = v->opp[a];
        double Sa, Sb;
        guo_source(v, a, u, Fn, &Sa);
        guo_source(v, b, u, Fn, &Sb);
        double fp = 0.5 * (fn[a] + fn[b]), fm = 0.5 * (fn[a] - fn[b]);
        double ep = 0.5 * (feq[a] + feq[b]), em = 0.5 * (feq[a] - feq[b]);
        double sp = 0.5 * (Sa + Sb), sm = 0.5 * (Sa - Sb);
        out[a] = fn[a] - m->omega * (fp - ep) - m->omega_m * (fm - em)
                 + (1.0 - 0.5 * m->omega) * sp + (1.0 - 0.5 * m->omega_m) * sm;
    }
}

/* MRT collision (not in the paper): overwrites out[] with
 *     f*_a = f_a - sum_k M_ka [s_k m_k(f - feq) - (1 - s_k/2) m_k(S)] / |M_k|^2. */
static void collide_node_mrt(const or_model *m, const double *fn, const double *Fn,
                             const double *feq, const double u[3], double *out)
{
    const or_dvm *v = &m->v;
    double S[OR_MAXQ];
    for (int a = 0; a < v->Q; ++a)
        guo_source(v, a, u, Fn, &S[a]);
    for (int a = 0; a < v->Q; ++a)
        out[a] = fn[a];
    for (int k = 0; k < m->nrow; ++k) {
        double mn = 0.0, mS = 0.0;
        for (int a = 0; a < v->Q; ++a) {
            mn += m->M[k][a] * (fn[a] - feq[a]);
            mS += m->M[k][a] * S[a];
        }
        const double ck = (m->s_row[k] * mn - (1.0 - 0.5 * m->s_row[k]) * mS) / m->M2[k];
        for (int a = 0; a < v->Q; ++a)
            out[a] -= ck * m->M[k][a];
    }
}

/* The MRT moment basis and the rate of each row (see the header): monomials
 * of degree 0, 1, 2 (|e|^2 first), 3, ... with exponents up to 2,
 * orthogonalised over the velocity set in that order. */
static int build_mrt(or_model *m, double s_bulk, double s_even, double s_odd)
{
    const or_dvm *v = &m->v;
    const int D = v->d;
    m->nrow = 0;
    for (int deg = 0; deg <= 2 * D; ++deg) {
        /* candidate vectors of this degree; code -1 = |e|^2 */
        int npow = 1;
        for (int k = 0; k < D; ++k)
            npow *= 3;
        for (int c = (deg == 2 ? -1 : 0); c < npow; ++c) {
            int pw[3] = {0, 0, 0}, sum = 0;
            if (c >= 0) {
                int r = c;
                for (int k = 0; k < D; ++k) {
                    pw[k] = r % 3;
                    r /= 3;
                    sum += pw[k];
                }
                if (sum != deg)
                    continue;
            }
            double w[OR_MAXQ];
            for (int a = 0; a < v->Q; ++a) {
                if (c < 0) {
                    w[a] = 0.0;
                    for (int k = 0; k < D; ++k)
                        w[a] += v->e[a][k] * v->e[a][k];
                } else {
                    w[a] = 1.0;
                    for (int k = 0; k < D; ++k)
                        for (int i = 0; i < pw[k]; ++i)
                            w[a] *= v->e[a][k];
                }
            }
            for (int r = 0; r < m->nrow; ++r) {
                double dot = 0.0;
                for (int a = 0; a < v->Q; ++a)
                    dot += w[a] * m->M[r][a];
                for (int a = 0; a < v->Q; ++a)
                    w[a] -= dot / m->M2[r] * m->M[r][a];
            }
            double n2 = 0.0;
            for (int a = 0; a < v->Q; ++a)
                n2 += w[a] * w[a];
            if (n2 < 1e-9)
                continue; /* dependent on the rows so far */
            if (m->nrow >= v->Q)
                return OR_ERR_ARG;
            for (int a = 0; a < v->Q; ++a)
                m->M[m->nrow][a] = w[a];
            m->M2[m->nrow] = n2;
            m->s_row[m->nrow] = deg <= 1    ? m->omega
                                : c < 0     ? s_bulk
                                : deg == 2  ? m->omega
                                : deg % 2   ? s_odd
                                            : s_even;
            ++m->nrow;
        }
    }
    return m->nrow == v->Q ? OR_OK : OR_ERR_ARG;
}

/* Eq. (collision): f*_a = f_a - omega (f_a - feq_a), omega = 1/(tau_p + 1/2)
 * = 1/tau_std, plus the Guo source in the same trapezoidal form. */
static void collide_node(const or_model *m, const double *fn, const double *Fn,
                         double *out)
{
    const or_dvm *v = &m->v;
    double P, u[3], feq[OR_MAXQ];
    node_moments(m, fn, Fn, &P, u);
    equilibrium(v, m->compressible, m->rho0, P, u, feq);
    double src_fac = 1.0 - 0.5 * m->omega;
    for (int a = 0; a < v->Q; ++a) {
        double S = 0.0;
        if (Fn) {
            double eu = v->e[a][0] * u[0] + v->e[a][1] * u[1] + v->e[a][2] * u[2];
            double eF = v->e[a][0] * Fn[0] + v->e[a][1] * Fn[1] + v->e[a][2] * Fn[2];
            double uF = u[0] * Fn[0] + u[1] * Fn[1] + u[2] * Fn[2];
            S = v->t[a] * ((eF - uF) * INV_CS2 + eu * eF * INV_CS2 * INV_CS2);
        }
        out[a] = fn[a] - m->omega * (fn[a] - feq[a]) + src_fac * S;
    }
    if (m->omega_m > 0.0)
        collide_node_trt(m, fn, Fn, feq, u, out);
    else if (m->mrt)
        collide_node_mrt(m, fn, Fn, feq, u, out);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1 Eq. (propagation) with Sec. 2.2 Eq. (bb).                        */

/* Upstream node of x along -e_a.  Returns 1 and the node index when it lies in
 * the domain (after periodic wrap), 0 when it lies beyond a wall; *on_lid is
 * set when that wall is the +y face (upstream y >= ny). */
static int upstream(const or_model *m, int x, int y, int z, const int e[3], long *n_up,
                    int *on_lid)
{
    int c[3] = {x - e[0], y - e[1], z - e[2]};
    int L[3] = {m->nx, m->ny, m->nz};
    int inside = 1;
    *on_lid = 0;
    for (int k = 0; k < 3; ++k) {
        if (c[k] < 0 || c[k] >= L[k]) {
            if (m->periodic[k])
                c[k] = (c[k] + L[k]) % L[k];
            else
                inside = 0;
        }
    }
    if (!inside) {
        *on_lid = m->lid_on && (y - e[1] >= m->ny);
        return 0;
    }
    *n_up = (long)c[0] + (long)m->nx * ((long)c[1] + (long)m->ny * c[2]);
    return 1;
}

static long node_index(const or_model *m, int x, int y, int z)
{
    return (long)x + (long)m->nx * ((long)y + (long)m->ny * z);
}

static int is_solid(const or_model *m, long n) { return m->solid && m->solid[n]; }

/* Velocity of the inlet face at the face position of node (x, y, z); the
 * face's nodes are numbered by the two remaining axes, lower axis fastest. */
static void inlet_velocity(const or_model *m, int x, int y, int z, double U[3])
{
    int f = -1;
    for (int i = 0; i < 6; ++i)
        if (m->face[i] == OR_FACE_INLET)
            f = i;
    long idx, nf;
    if (f / 2 == 0) {
        idx = y + (long)m->ny * z;
        nf = (long)m->ny * m->nz;
    } else if (f / 2 == 1) {
        idx = x + (long)m->nx * z;
        nf = (long)m->nx * m->nz;
    } else {
        idx = x + (long)m->nx * y;
        nf = (long)m->nx * m->ny;
    }
    U[0] = U[1] = U[2] = 0.0;
    for (int k = 0; k < m->v.d; ++k)
        U[k] = m->inlet_u[k * nf + idx];
}

/* Where the population entering fluid node (x, y, z) along e_a comes from
 * (the rule in the header): OR_LINK_STREAM with the source node and slot,
 * or a bounce (OR_LINK_WALL, OR_LINK_SOLID, OR_LINK_OUTFLOW) involving slot
 * abar of the node itself, with *term the moving-wall term of a wall or
 * inlet link. */
static int resolve_link_at(const or_model *m, int x, int y, int z, int a, long *src, int *slot,
                           double *term, int nested);

static int resolve_link(const or_model *m, int x, int y, int z, int a, long *src, int *slot,
                        double *term)
{
    return resolve_link_at(m, x, y, z, a, src, slot, term, 0);
}

/* nested: resolving the opposite population for a nodal link (a nodal
 * crossing there reports OR_LINK_NODAL without looking further). */
static int resolve_link_at(const or_model *m, int x, int y, int z, int a, long *src, int *slot,
                           double *term, int nested)
{
    const or_dvm *v = &m->v;
    const int c[3] = {x, y, z}, L[3] = {m->nx, m->ny, m->nz};
    int up[3], e[3], bounce = 0, inlet = 0, lid = 0, outflow = 0, nodal = 0;
    for (int k = 0; k < 3; ++k) {
        e[k] = v->e[a][k];
        up[k] = c[k] - e[k];
        if (up[k] >= 0 && up[k] < L[k])
            continue;
        int face = 2 * k + (up[k] >= L[k] ? 1 : 0);
        switch (m->face[face]) {
        case OR_FACE_PERIODIC:
            up[k] = (up[k] + L[k]) % L[k];
            break;
        case OR_FACE_WALL:
            bounce = 1;
            if (face == 3)
                lid = m->lid_on;
            break;
        case OR_FACE_INLET:
            bounce = 1;
            inlet = 1;
            break;
        case OR_FACE_OUTFLOW:
            outflow = 1;
            break;
        case OR_FACE_NODAL:
            nodal = 1;
            if (face == 3)
                lid = m->lid_on;
            break;
        case OR_FACE_SYMMETRY:
            up[k] = c[k];
            e[k] = -e[k];
            break;
        }
    }
    *term = 0.0;
    if (bounce || nodal) {
        double U[3] = {0.0, 0.0, 0.0};
        if (inlet)
            inlet_velocity(m, x, y, z, U);
        else if (lid)
            for (int k = 0; k < 3; ++k)
                U[k] = m->lid[k];
        double eU = v->e[a][0] * U[0] + v->e[a][1] * U[1] + v->e[a][2] * U[2];
        *term = 2.0 * v->t[a] * m->rho0 * eU * INV_CS2;
        *src = node_index(m, x, y, z);
        *slot = v->opp[a];
        if (bounce)
            return OR_LINK_WALL;
        if (!nested) { /* nodal: the opposite population that has just arrived */
            long s2;
            int sl2;
            double t2;
            if (resolve_link_at(m, x, y, z, v->opp[a], &s2, &sl2, &t2, 1) == OR_LINK_STREAM) {
                *src = s2;
                *slot = sl2;
            }
        }
        return OR_LINK_NODAL;
    }
    if (outflow) {
        *src = node_index(m, x, y, z);
        *slot = v->opp[a];
        return OR_LINK_OUTFLOW;
    }
    long nu = node_index(m, up[0], up[1], up[2]);
    if (is_solid(m, nu)) {
        *src = node_index(m, x, y, z);
        *slot = v->opp[a];
        return OR_LINK_SOLID;
    }
    /* the (possibly reflected) direction e */
    int b = a;
    if (e[0] != v->e[a][0] || e[1] != v->e[a][1] || e[2] != v->e[a][2])
        for (int i = 0; i < v->Q; ++i)
            if (v->e[i][0] == e[0] && v->e[i][1] == e[1] && v->e[i][2] == e[2])
                b = i;
    *src = nu;
    *slot = b;
    return OR_LINK_STREAM;
}

/* Velocity of node n from its post-collision populations: collision keeps P
 * and adds F to j, so u = (sum e fb - F/2)/rho. */
static void post_collision_velocity(const or_model *m, const double *fb, long n, double u[3])
{
    const or_dvm *v = &m->v;
    double s = 0.0, j[3] = {0.0, 0.0, 0.0}, Fn[3];
    load_force(m, n, Fn);
    for (int a = 0; a < v->Q; ++a) {
        s += fb[n * v->Q + a];
        for (int k = 0; k < 3; ++k)
            j[k] += v->e[a][k] * fb[n * v->Q + a];
    }
    double rho = m->compressible ? s : m->rho0;
    for (int k = 0; k < 3; ++k)
        u[k] = (j[k] - 0.5 * Fn[k]) / rho;
}

/* Even half of the equilibrium, feq+_a(P, u) = (feq_a + feq_abar)/2. */
static double equilibrium_even(const or_model *m, int a, double P, const double u[3])
{
    double feq[OR_MAXQ];
    equilibrium(&m->v, m->compressible, m->rho0, P, u, feq);
    return 0.5 * (feq[a] + feq[m->v.opp[a]]);
}

/* BoundaryCondition + Propagation: fb (post-collision) -> f (post-propagation)
 * at every fluid node, each population taken where resolve_link says. */
static void propagate(const or_model *m, const double *fb, double *f)
{
    const or_dvm *v = &m->v;
    const int Q = v->Q;
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < m->nz; ++z)
        for (int y = 0; y < m->ny; ++y)
            for (int x = 0; x < m->nx; ++x) {
                long n = node_index(m, x, y, z);
                if (is_solid(m, n))
                    continue;
                for (int a = 0; a < Q; ++a) {
                    long src;
                    int slot;
                    double term;
                    int kind = resolve_link(m, x, y, z, a, &src, &slot, &term);
                    if (kind == OR_LINK_OUTFLOW) {
                        double u[3];
                        post_collision_velocity(m, fb, n, u);
                        f[n * Q + a] = -fb[n * Q + v->opp[a]] +
                                       2.0 * equilibrium_even(m, a, m->P_out, u);
                    } else {
                        f[n * Q + a] = fb[src * Q + slot] + term;
                    }
                }
            }
}

/* Momentum exchange (Sec. 5): force on the solid nodes during the
 * propagation fb -> f, sum over fluid nodes x and links a whose source is an
 * obstacle of 2 fb_abar(x) e_abar (the population leaving x towards the
 * solid and coming back reversed).  Each z-plane is summed in a fixed order
 * (planes in parallel), then the planes in order: the result does not
 * depend on the thread count. */
static void obstacle_force(const or_model *m, const double *fb, double out[3])
{
    const or_dvm *v = &m->v;
    const int Q = v->Q;
    double *plane = calloc((size_t)m->nz * 3, sizeof(double));
    out[0] = out[1] = out[2] = 0.0;
    if (!plane)
        return;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < m->nz; ++z)
        for (int y = 0; y < m->ny; ++y)
            for (int x = 0; x < m->nx; ++x) {
                long n = node_index(m, x, y, z);
                if (is_solid(m, n))
                    continue;
                for (int a = 0; a < Q; ++a) {
                    long src;
                    int slot;
                    double term;
                    if (resolve_link(m, x, y, z, a, &src, &slot, &term) != OR_LINK_SOLID)
                        continue;
                    int b = v->opp[a];
                    for (int k = 0; k < 3; ++k)
                        plane[3 * z + k] += 2.0 * fb[n * Q + b] * v->e[b][k];
                }
            }
    for (int z = 0; z < m->nz; ++z)
        for (int k = 0; k < 3; ++k)
            out[k] += plane[3 * z + k];
    free(plane);
}

static void collide_all(const or_model *m, const double *f, double *fb)
{
    const int Q = m->v.Q;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < m->N; ++n) {
        if (is_solid(m, n))
            continue;
        double Fn[3];
        load_force(m, n, Fn);
        collide_node(m, f + n * Q, m->F ? Fn : NULL, fb + n * Q);
    }
}

/* PostProcessing: p = c_s^2 P and u at every node (SoA outputs). */
static void postprocess(const or_model *m, const double *f, double *p_out, double *u_out)
{
    const int Q = m->v.Q;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < m->N; ++n) {
        double Fn[3], P, u[3];
        load_force(m, n, Fn);
        node_moments(m, f + n * Q, m->F ? Fn : NULL, &P, u);
        if (is_solid(m, n))
            P = u[0] = u[1] = u[2] = 0.0;
        if (p_out)
            p_out[n] = P / INV_CS2;
        if (u_out)
            for (int k = 0; k < m->v.d; ++k)
                u_out[(long)k * m->N + n] = u[k];
    }
}

/* Sec. 2.2: f = feq(p0, u0) at every node. */
static void init_equilibrium(const or_model *m, const double *p0, const double *u0, double *f)
{
    const int Q = m->v.Q;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < m->N; ++n) {
        double P = (p0 ? p0[n] : 1.0 / INV_CS2) * INV_CS2;
        double u[3] = {0.0, 0.0, 0.0};
        if (u0)
            for (int k = 0; k < m->v.d; ++k)
                u[k] = u0[(long)k * m->N + n];
        equilibrium(&m->v, m->compressible, m->rho0, P, u, f + n * Q);
    }
}

/* The three named box types as face types. */
static int faces_of_bc(int bc, int faces[6])
{
    if (bc != OR_BC_PERIODIC && bc != OR_BC_CAVITY && bc != OR_BC_CHANNEL)
        return OR_ERR_ARG;
    for (int k = 0; k < 3; ++k) {
        int periodic = (k == 1) ? (bc == OR_BC_PERIODIC) : (bc != OR_BC_CAVITY);
        faces[2 * k] = faces[2 * k + 1] = periodic ? OR_FACE_PERIODIC : OR_FACE_WALL;
    }
    return OR_OK;
}

static int setup_model(or_model *m, int lattice, int nx, int ny, int nz, double tau,
                       const int faces[6], int compressible, double rho0, const double *lid,
                       const double *F, double trt_lambda, const double *mrt)
{
    memset(m, 0, sizeof(*m));
    if (build_dvm(lattice, &m->v) != OR_OK)
        return OR_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || !(tau > 0.5) || !(rho0 > 0.0))
        return OR_ERR_ARG;
    if (m->v.d == 2 && nz != 1)
        return OR_ERR_ARG;
    int ninlet = 0;
    for (int i = 0; i < 6; ++i) {
        if (faces[i] < OR_FACE_PERIODIC || faces[i] > OR_FACE_NODAL)
            return OR_ERR_ARG;
        /* periodic faces come in pairs */
        if ((faces[i] == OR_FACE_PERIODIC) != (faces[i ^ 1] == OR_FACE_PERIODIC))
            return OR_ERR_ARG;
        /* 2D: no direction leaves through a z face */
        m->face[i] = (m->v.d == 2 && i >= 4) ? OR_FACE_PERIODIC : faces[i];
        ninlet += m->face[i] == OR_FACE_INLET;
    }
    if (ninlet > 1)
        return OR_ERR_ARG;
    m->nx = nx;
    m->ny = ny;
    m->nz = nz;
    m->N = (long)nx * ny * nz;
    for (int k = 0; k < 3; ++k)
        m->periodic[k] = m->face[2 * k] == OR_FACE_PERIODIC;
    m->lid_on = m->face[3] == OR_FACE_WALL || m->face[3] == OR_FACE_NODAL;
    for (int k = 0; k < 3; ++k)
        m->lid[k] = lid ? lid[k] : 0.0;
    m->omega = 1.0 / tau;
    if (!(trt_lambda >= 0.0))
        return OR_ERR_ARG;
    if (trt_lambda > 0.0) /* Lambda = (tau - 1/2)(1/omega_m - 1/2) */
        m->omega_m = 1.0 / (trt_lambda / (tau - 0.5) + 0.5);
    m->rho0 = rho0;
    m->compressible = compressible;
    m->F = F;
    if (mrt) { /* rates s_bulk, s_even, s_odd in (0, 2); not with TRT */
        for (int k = 0; k < 3; ++k)
            if (!(mrt[k] > 0.0 && mrt[k] < 2.0))
                return OR_ERR_ARG;
        if (trt_lambda > 0.0)
            return OR_ERR_ARG;
        m->mrt = 1;
        if (build_mrt(m, mrt[0], mrt[1], mrt[2]) != OR_OK)
            return OR_ERR_ARG;
    }
    return OR_OK;
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* Exported: the forward run.
 *   p0 (N) / u0 (d*N): initial pressure and velocity, NULL = 1/3 and 0.
 *   F (d*N): body force or NULL.  lid (3): moving-wall velocity or NULL.
 *   After nsteps steps of Sec. 3.1's loop, writes p (N), u (d*N) and, when
 *   f_out is given, the post-propagation distributions f (Q*N,
 *   direction-major). */
int or_run_faces(int lattice, int nx, int ny, int nz, double tau, const int *faces,
                 int compressible, double rho0, const double *lid, const double *F,
                 const unsigned char *solid, const double *inlet_u, const double *p0,
                 const double *u0, double p_outflow, long nsteps, double *p_out,
                 double *u_out, double *f_out, double *force_out, int nthreads,
                 double trt_lambda, const double *mrt)
{
    or_model m;
    int rc = setup_model(&m, lattice, nx, ny, nz, tau, faces, compressible, rho0, lid, F,
                         trt_lambda, mrt);
    if (rc != OR_OK || nsteps < 0)
        return OR_ERR_ARG;
    int has_inlet = 0;
    for (int i = 0; i < 6; ++i)
        has_inlet |= m.face[i] == OR_FACE_INLET;
    if (has_inlet && !inlet_u)
        return OR_ERR_ARG;
    m.solid = solid;
    m.inlet_u = inlet_u;
    m.P_out = p_outflow * INV_CS2;
    set_threads(nthreads);
    const int Q = m.v.Q;
    double *f = malloc(sizeof(double) * Q * m.N);
    double *fb = malloc(sizeof(double) * Q * m.N);
    if (!f || !fb) {
        free(f);
        free(fb);
        return OR_ERR_NOMEM;
    }
    init_equilibrium(&m, p0, u0, f);
    if (force_out)
        force_out[0] = force_out[1] = force_out[2] = 0.0;
    for (long it = 0; it < nsteps; ++it) {
        collide_all(&m, f, fb);   /* Collision */
        if (force_out && it == nsteps - 1)
            obstacle_force(&m, fb, force_out);
        propagate(&m, fb, f);     /* BoundaryCondition + Propagation */
    }
    postprocess(&m, f, p_out, u_out); /* PostProcessing */
    if (f_out)
        for (long n = 0; n < m.N; ++n)
            for (int a = 0; a < Q; ++a)
                f_out[(long)a * m.N + n] = f[n * Q + a];
    free(f);
    free(fb);
    return OR_OK;
}

/* Exported: or_run_faces for the three named box types (no obstacles). */
int or_run(int lattice, int nx, int ny, int nz, double tau, int bc, int compressible,
           double rho0, const double *lid, const double *F, const double *p0,
           const double *u0, long nsteps, double *p_out, double *u_out, double *f_out,
           int nthreads, double trt_lambda, const double *mrt)
{
    int faces[6];
    if (faces_of_bc(bc, faces) != OR_OK)
        return OR_ERR_ARG;
    return or_run_faces(lattice, nx, ny, nz, tau, faces, compressible, rho0, lid, F, NULL,
                        NULL, p0, u0, 1.0 / INV_CS2, nsteps, p_out, u_out, f_out, NULL,
                        nthreads, trt_lambda, mrt);
}

/* Exported: one collision at one node (tiny brute-force pins). */
int or_collide_node(int lattice, double tau, int compressible, double rho0, const double *fn,
                    const double *F3, double *out, double trt_lambda, const double *mrt)
{
    or_model m;
    int faces[6] = {0, 0, 0, 0, 0, 0};
    int rc = setup_model(&m, lattice, 1, 1, 1, tau, faces, compressible, rho0, NULL, NULL,
                         trt_lambda, mrt);
    if (rc != OR_OK)
        return rc;
    collide_node(&m, fn, F3, out);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Adjoint (not in the paper).  One step maps the pre-collision field f^k to
 * f^{k+1} = S(C(f^k)), with C the collision above and S the bounce-back +
 * propagation map, affine in the lid velocity U.  With
 *     J = rho0/2 sum_x |u(f^T)(x)|^2,
 * lambda^T_a(x) = dJ/df^T_a(x) = e_a . u^T(x), and going backwards
 *     mu^k     = S^T lambda^{k+1},
 *     lambda^k = (dC/df at f^k)^T mu^k,
 *     dJ/dF   += (dC/dF at f^k)^T mu^k,     dJ/dU += (dS/dU)^T lambda^{k+1},
 * plus the direct term dJ/dF = u^T/2 from u = (j + F/2)/rho0.  The Jacobian
 * of C is formed entry by entry below from the definitions, incompressible
 * model only.  States are kept every K steps and recomputed in between. */

/* Jacobian of collide_node at one node: Jf[a*Q+b] = d f*_a / d f_b and
 * JF[a*3+i] = d f*_a / d F_i. */
static void collide_jacobian(const or_model *m, const double *fn, const double *Fn,
                             double *Jf, double *JF)
{
    const or_dvm *v = &m->v;
    const int Q = v->Q;
    const double w = m->omega, r0 = m->rho0;
    double P, u[3];
    node_moments(m, fn, Fn, &P, u);
    double F[3] = {Fn ? Fn[0] : 0.0, Fn ? Fn[1] : 0.0, Fn ? Fn[2] : 0.0};
    for (int a = 0; a < Q; ++a) {
        const int *ea = v->e[a];
        double eu = ea[0] * u[0] + ea[1] * u[1] + ea[2] * u[2];
        double eF = ea[0] * F[0] + ea[1] * F[1] + ea[2] * F[2];
        /* d feq_a / d u_i   = t_a rho0 (3 e_i + 9 (e.u) e_i - 3 u_i)
         * d S_a  / d u_i    = t_a (-3 F_i + 9 (e.F) e_i)
         * d S_a  / d F_i    = t_a (3 (e_i - u_i) + 9 (e.u) e_i)
         * d P    / d f_b    = 1,  d u_i / d f_b = e_b,i / rho0,
         * d u_i  / d F_j    = delta_ij / (2 rho0). */
        double dfeq_du[3], dS_du[3], dS_dF[3];
        for (int i = 0; i < 3; ++i) {
            dfeq_du[i] = v->t[a] * r0 *
                         (ea[i] * INV_CS2 + eu * ea[i] * INV_CS2 * INV_CS2 - u[i] * INV_CS2);
            dS_du[i] = v->t[a] * (-F[i] * INV_CS2 + eF * ea[i] * INV_CS2 * INV_CS2);
            dS_dF[i] = v->t[a] * ((ea[i] - u[i]) * INV_CS2 + eu * ea[i] * INV_CS2 * INV_CS2);
        }
        for (int b = 0; b < Q; ++b) {
            const int *eb = v->e[b];
            double du_dfb[3] = {eb[0] / r0, eb[1] / r0, eb[2] / r0};
            double dfeq = v->t[a] * 1.0; /* through P */
            double dS = 0.0;
            for (int i = 0; i < 3; ++i) {
                dfeq += dfeq_du[i] * du_dfb[i];
                dS += dS_du[i] * du_dfb[i];
            }
            Jf[a * Q + b] = (a == b ? 1.0 - w : 0.0) + w * dfeq + (1.0 - 0.5 * w) * dS;
        }
        for (int i = 0; i < 3; ++i) {
            double du_dFi = 0.5 / r0;
            JF[a * 3 + i] = w * dfeq_du[i] * du_dFi +
                            (1.0 - 0.5 * w) * (dS_dF[i] + dS_du[i] * du_dFi);
        }
    }
}

/* mu = S^T lambda, and the lid-velocity gradient.  S sends fb_a(y) to
 * f_a(y + e_a) when that node's upstream is y, and fb_abar(x) to f_a(x) when
 * x's upstream along -e_a is beyond a wall.  So mu_a(y) collects exactly one
 * entry: lambda_a(y + e_a) in the first case, lambda_abar(y) in the second.
 * Written here as a scatter over (x, a) that mirrors propagate(). */
static void propagate_transpose(const or_model *m, const double *lam, double *mu, double gU[3])
{
    const or_dvm *v = &m->v;
    const int Q = v->Q;
    memset(mu, 0, sizeof(double) * Q * m->N);
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (int z = 0; z < m->nz; ++z)
        for (int y = 0; y < m->ny; ++y)
            for (int x = 0; x < m->nx; ++x) {
                long n = (long)x + (long)m->nx * ((long)y + (long)m->ny * z);
                for (int a = 0; a < Q; ++a) {
                    long nu;
                    int lid;
                    double l = lam[n * Q + a];
                    if (upstream(m, x, y, z, v->e[a], &nu, &lid)) {
                        mu[nu * Q + a] += l;
                    } else {
                        mu[n * Q + v->opp[a]] += l;
                        if (lid) {
                            double c = 2.0 * v->t[a] * m->rho0 * INV_CS2 * l;
                            g0 += c * v->e[a][0];
                            g1 += c * v->e[a][1];
                            g2 += c * v->e[a][2];
                        }
                    }
                }
            }
    gU[0] += g0;
    gU[1] += g1;
    gU[2] += g2;
}

/* lambda = (dC/df)^T mu at every node; gF += (dC/dF)^T mu. */
static void collide_transpose(const or_model *m, const double *f, const double *mu,
                              double *lam, double *gF)
{
    const int Q = m->v.Q;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < m->N; ++n) {
        double Fn[3], Jf[OR_MAXQ * OR_MAXQ], JF[OR_MAXQ * 3];
        load_force(m, n, Fn);
        collide_jacobian(m, f + n * Q, m->F ? Fn : NULL, Jf, JF);
        for (int b = 0; b < Q; ++b) {
            double s = 0.0;
            for (int a = 0; a < Q; ++a)
                s += mu[n * Q + a] * Jf[a * Q + b];
            lam[n * Q + b] = s;
        }
        for (int i = 0; i < m->v.d; ++i) {
            double s = 0.0;
            for (int a = 0; a < Q; ++a)
                s += mu[n * Q + a] * JF[a * 3 + i];
            gF[(long)i * m->N + n] += s;
        }
    }
}

/* Exported: J and its gradients after T steps (incompressible model).
 *   dJdF (d*N, component-major) and dJdU (3) are overwritten.  K is the
 *   checkpoint interval (1 <= K).  Same inputs as or_run. */
int or_adjoint(int lattice, int nx, int ny, int nz, double tau, int bc, double rho0,
               const double *lid, const double *F, const double *p0, const double *u0,
               long T, long K, double *J_out, double *dJdF, double *dJdU, int nthreads)
{
    or_model m;
    int faces[6];
    if (faces_of_bc(bc, faces) != OR_OK)
        return OR_ERR_ARG;
    int rc = setup_model(&m, lattice, nx, ny, nz, tau, faces, 0, rho0, lid, F, 0.0, NULL);
    if (rc != OR_OK || T < 1 || K < 1)
        return OR_ERR_ARG;
    set_threads(nthreads);
    const int Q = m.v.Q, d = m.v.d;
    const long N = m.N, QN = (long)Q * N;
    long nseg = (T + K - 1) / K;
    double *ckpt = malloc(sizeof(double) * QN * nseg);
    double *seg = malloc(sizeof(double) * QN * K);
    double *fb = malloc(sizeof(double) * QN);
    double *lam = malloc(sizeof(double) * QN);
    double *mu = malloc(sizeof(double) * QN);
    double *fT = malloc(sizeof(double) * QN);
    if (!ckpt || !seg || !fb || !lam || !mu || !fT) {
        free(ckpt); free(seg); free(fb); free(lam); free(mu); free(fT);
        return OR_ERR_NOMEM;
    }
    /* forward, keeping f^{sK} */
    init_equilibrium(&m, p0, u0, fT);
    for (long k = 0; k < T; ++k) {
        if (k % K == 0)
            memcpy(ckpt + (k / K) * QN, fT, sizeof(double) * QN);
        collide_all(&m, fT, fb);
        propagate(&m, fb, fT);
    }
    /* objective and seed */
    double J = 0.0;
    for (long i = 0; i < (long)d * N; ++i)
        dJdF[i] = 0.0;
    for (long n = 0; n < N; ++n) {
        double Fn[3], P, u[3];
        load_force(&m, n, Fn);
        node_moments(&m, fT + n * Q, m.F ? Fn : NULL, &P, u);
        J += 0.5 * rho0 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        for (int a = 0; a < Q; ++a)
            lam[n * Q + a] = m.v.e[a][0] * u[0] + m.v.e[a][1] * u[1] + m.v.e[a][2] * u[2];
        for (int i = 0; i < d; ++i)
            dJdF[(long)i * N + n] = 0.5 * u[i]; /* direct: du/dF = 1/(2 rho0) */
    }
    double gU[3] = {0.0, 0.0, 0.0};
    /* backward over segments */
    for (long s = nseg - 1; s >= 0; --s) {
        long k0 = s * K, k1 = (k0 + K < T) ? k0 + K : T;
        memcpy(seg, ckpt + s * QN, sizeof(double) * QN);
        for (long k = k0 + 1; k < k1; ++k) {
            collide_all(&m, seg + (k - 1 - k0) * QN, fb);
            propagate(&m, fb, seg + (k - k0) * QN);
        }
        for (long k = k1 - 1; k >= k0; --k) {
            propagate_transpose(&m, lam, mu, gU);
            collide_transpose(&m, seg + (k - k0) * QN, mu, lam, dJdF);
        }
    }
    *J_out = J;
    for (int i = 0; i < 3; ++i)
        dJdU[i] = gU[i];
    free(ckpt); free(seg); free(fb); free(lam); free(mu); free(fT);
    return OR_OK;
}
