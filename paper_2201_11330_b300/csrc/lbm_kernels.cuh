// lbm_kernels.cuh -- fused stream-collide, initialisation and moment kernels.
//
// One launch of k_step is one IMEXLBM time step (arxiv 2201.11330, Sec. 3.1:
// Collision -> BoundaryCondition -> Propagation -> PostProcessing), fused:
// each thread owns one node, gathers its Q incoming populations (propagation,
// Eq. (propagation), with half-way bounce-back, Eq. (bb), and the moving-lid
// term at walls, index wrap at periodic faces), takes the moments (Sec. 2.1),
// relaxes towards the incompressible equilibrium of Eq. (incompressible_feq)
// (or Eq. (feq)) with the IMEX factor omega = 1/(tau_paper + 1/2) of Eq.
// (collision), and stores the post-collision populations.  The stored state
// is therefore always post-collision; moments are computed from it on demand.
//
// Layout in HBM: structure of arrays, slot a of node n at f[a*N + n], node
// index n = x + nx*(y + ny*z), x fastest.  Three access patterns:
//   PAT_PULL   two lattices: read slot a of the upstream node x - e_a from
//              `src`, write slot a of x to `dst`.
//   PAT_GATHER single lattice (AA pattern, first half): read slot abar of
//              x - e_a, write slot a of x + e_a (in place).
//   PAT_LOCAL  single lattice (AA pattern, second half): read slot a of x,
//              write slot abar of x (in place).
// A thread of PAT_GATHER reads exactly the locations it writes, so the
// in-place update is race-free without synchronisation.
#pragma once

#include "lbm_lattice.cuh"

namespace lbm {

enum Pattern { PAT_PULL = 0, PAT_GATHER = 1, PAT_LOCAL = 2 };
// Collision model of a step kernel: incompressible BGK (the paper's),
// compressible BGK, incompressible two-relaxation-time.
enum Model { M_INC = 0, M_COMP = 1, M_TRT = 2, M_MRT = 3 };
// Where post-collision populations f*_a(x) sit in the stored state.
enum Form { FORM_LOCAL = 0, FORM_SWAPPED = 1, FORM_STREAMED = 2 };

constexpr int kMaxQ = 27;
constexpr int kReduceVals = 6;  // sum dP, momentum x/y/z, kinetic energy, max |u|^2
constexpr int kPartialStride = 8;
constexpr int kMonSlots = 256;  // threads of the largest block (monitor columns)

template <class R>
struct Coef {
    R omega;     // 1/tau (standard tau)
    R rho0;      // constant density of the incompressible model
    R inv_rho0;  // 1/rho0
    R sigma;     // 1 when the storage holds f - t, else 0
    R kf;        // (1 - omega/2)/omega: force source folded into the equilibrium
    R omega_m;   // TRT: relaxation rate of the antisymmetric part
    R kf_m;      // TRT: (1 - omega_m/2)/omega_m
    R lid[kMaxQ];  // 2 t_a rho0 (e_a . U)/c_s^2 for links crossing the moving wall
    R mrt[3];      // MRT: rates of the bulk, even and odd higher moments
    R pout2;       // outflow: 2 (P_out - sigma)
    R pout_r;      // outflow: density of the even equilibrium (rho0, or P_out if compressible)
};

struct StepParams {
    int nx, ny, nz;
    int N;
    int periodic;  // bit k set: axis k is periodic, else walled
    int lid_on;    // the +y wall moves
    Coef<float> cf;
    Coef<double> cd;
    // per-face boundaries and obstacles (general kernel, lbm_geo.cuh)
    int face[6];            // lbm_face per face: -x, +x, -y, +y, -z, +z
    const unsigned *links;  // per-node link word, or NULL (no obstacles)
    const float *inlet;     // inlet velocity, d * (face nodes), or NULL (at rest)
    int inlet_face;         // face index of the inlet, or -1
    const int *nlist;       // general kernel on a node list: the nodes, or NULL (full grid)
    int nlist_len;          // entries of nlist
    long long part_base;    // node-list launches: first partial entry of their blocks
    int open_faces;         // bit f: face f is an inlet, outflow, symmetry or nodal face
    int xm;                 // node-list launches: the first / last xm nodes of every row
                            // next to an open x face go to the general kernel
    double *partials;  // per-block monitor sums (RED kernels)
    const float *F;  // body force, d*N component-major (FORCE kernels)
    void *u_out;     // velocity output, d*N component-major, kernel arithmetic type (UOUT)
    // Element offsets from node n, for rows with neighbours in y and z on both
    // sides: pull_off[a] = slot a of the row shifted by -e_a (a N - e_a,y nx -
    // e_a,z nx ny), push_off[a] = slot a of the row shifted by +e_a.  Uniform
    // across the grid, so an access costs one add to the node's address.
    long long pull_off[kMaxQ];
    long long push_off[kMaxQ];
    // push_off again, read by the AA push stores: a separate copy keeps the
    // compiler from holding the loads' offsets in registers across the collision
    long long push_st[kMaxQ];
};

template <class R>
__device__ __forceinline__ const Coef<R> &coef(const StepParams &p);
template <>
__device__ __forceinline__ const Coef<float> &coef<float>(const StepParams &p)
{
    return p.cf;
}
template <>
__device__ __forceinline__ const Coef<double> &coef<double>(const StepParams &p)
{
    return p.cd;
}

// ---- memory access ---------------------------------------------------------
template <class T>
__device__ __forceinline__ T ld(const T *p)
{
#ifdef LBM_STREAMING_HINTS
    return __ldcs(p);
#else
    return *p;
#endif
}
template <class T>
__device__ __forceinline__ void st(T *p, T v)
{
#ifdef LBM_STREAMING_HINTS
    __stcs(p, v);
#else
    *p = v;
#endif
}

// ---- explicitly rounded arithmetic ------------------------------------------
// The collision is inlined into several kernels (pull, AA halves, paired); to
// make all of them round identically, every multiply-add is written out: the
// _rn intrinsics are never fused or split by the compiler.
__device__ __forceinline__ float o_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float o_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float o_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float o_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double o_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double o_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double o_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double o_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// ---- collision (Sec. 2.1) ---------------------------------------------------
// g holds the populations (shifted by sigma*t_a when the storage is shifted);
// on return it holds the post-collision populations in the same shift.  The
// incompressible update is invariant under that shift, so only the
// compressible density rho = sum g + sigma sees it.  u returns the velocity
// (j + F/2)/rho.  The Guo source (1 - omega/2) S_a is folded into the
// equilibrium as kf*S_a, and opposite directions are handled in pairs:
//   feq_a = t_a [A + 4.5 rho (e.u)^2] +/- t_a 3 rho (e.u),
//   A = sum g - 1.5 rho u.u  (the sigma*t_a shift cancels).
// x t_a for the odd (momentum) part of the equilibrium: in FP32 with the
// weight split into hi + lo (see w_lo), in FP64 a plain product.
template <class L, int a, class R>
__device__ __forceinline__ R wmul(R x)
{
    if constexpr (std::is_same<R, float>::value)
        return o_fma(x, w_hi<L>(a), o_mul(x, w_lo<L>(a)));
    else
        return o_mul(x, R(L::w(a)));
}

// Multiple-relaxation-time collision (not in the paper; d'Humieres et al.
// 2002) on the moments of MrtBasis<L>:
//     g*_a = g_a - sum_k M_ka [s_k m_k(n) - (1 - s_k/2) m_k(S)] / |M_k|^2,
// n = g - feq (feq without the source), S the Guo source t_a [3 (e_a - u).F
// + 9 (e_a.u)(e_a.F)].  Summed over a complete orthogonal basis with every
// s_k = omega this is the BGK update, so
//     g* = BGK(g) + sum_k M_ka (omega - s_k) [m_k(n) + m_k(S)/2] / |M_k|^2
// over the rows whose rate differs from omega: the bulk and the higher rows
// (the stress relaxes at omega; density and momentum at any rate give the
// same result, omega here).  mrt_corrections returns those coefficients,
// computed from the pre-collision g; collide() applies them after its BGK
// pass.  With every rate equal to omega the corrections vanish exactly.
template <class L, int r>
__host__ __device__ constexpr int mrt_norm2()
{
    int n = 0;
    for (int a = 0; a < L::Q; ++a)
        n += MrtBasis<L>::M[r][a] * MrtBasis<L>::M[r][a];
    return n;
}
template <class L, class R, bool FORCE>
__device__ __forceinline__ void mrt_corrections(const R (&g)[L::Q], const R (&F)[3],
                                                const Coef<R> &c, R s, R rho, R ir,
                                                const R (&jf)[3], const R (&u)[3],
                                                R (&ck)[L::Q])
{
    using B = MrtBasis<L>;
    constexpr int Q = L::Q, H = Q / 2;
    const R uu = o_fma(u[2], u[2], o_fma(u[1], u[1], o_mul(u[0], u[0])));
    const R A = o_fma(o_mul(R(-1.5), rho), uu, s);
    const R r3 = o_mul(R(3), rho), r45 = o_mul(R(4.5), rho);
    R uF = R(0);
    if constexpr (FORCE)
        uF = o_fma(u[2], F[2], o_fma(u[1], F[1], o_mul(u[0], F[0])));
    const R m3uF = o_mul(R(-3), uF);
    // h = n + S/2, the only combination the corrections need
    R h[Q];
    SFor<0, H>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        constexpr int b = opp<L>(a);
        R ej = R(0), eF = R(0);
        (void)eF;
        SFor<0, 3>::run([&](auto K_) {
            constexpr int k = decltype(K_)::value;
            if constexpr (L::e(a, k) == 1) {
                ej = o_add(ej, jf[k]);
                if constexpr (FORCE)
                    eF = o_add(eF, F[k]);
            } else if constexpr (L::e(a, k) == -1) {
                ej = o_sub(ej, jf[k]);
                if constexpr (FORCE)
                    eF = o_sub(eF, F[k]);
            }
        });
        const R t = R(L::w(a));
        const R eu = o_mul(ej, ir);
        R sym = o_fma(o_mul(r45, eu), eu, A), asym = o_mul(r3, eu);
        if constexpr (FORCE) {  // feq - S/2: S/2 = t [(9 eu eF - 3 uF)/2 +- 3 eF/2]
            sym = o_fma(o_mul(R(-4.5), eu), eF, o_fma(R(-0.5), m3uF, sym));
            asym = o_fma(R(-1.5), eF, asym);
        }
        h[a] = o_sub(g[a], o_mul(t, o_add(sym, asym)));
        h[b] = o_sub(g[b], o_mul(t, o_sub(sym, asym)));
    });
    {
        R a0 = A;
        if constexpr (FORCE)
            a0 = o_fma(R(-0.5), m3uF, a0);
        h[H] = o_sub(g[H], o_mul(R(L::w(H)), a0));
    }
    SFor<L::D + 1, Q>::run([&](auto R_) {
        constexpr int r = decltype(R_)::value;
        constexpr int kind = B::kind[r];
        if constexpr (kind == 2) {  // the stress: at omega, no correction
            ck[r] = R(0);
        } else {
            R mh = R(0);
            SFor<0, Q>::run([&](auto A_) {
                constexpr int a = decltype(A_)::value;
                constexpr int m = B::M[r][a];
                if constexpr (m == 1)
                    mh = o_add(mh, h[a]);
                else if constexpr (m == -1)
                    mh = o_sub(mh, h[a]);
                else if constexpr (m != 0)
                    mh = o_fma(R(m), h[a], mh);
            });
            const R rate = kind == 1 ? c.mrt[0] : kind == 3 ? c.mrt[1] : c.mrt[2];
            ck[r] = o_mul(o_mul(o_sub(c.omega, rate), mh), R(1.0 / mrt_norm2<L, r>()));
        }
    });
}

// g_a += sum_k M_ka ck_k over the rows that carry a correction.
template <class L, class R>
__device__ __forceinline__ void mrt_apply(R (&g)[L::Q], const R (&ck)[L::Q])
{
    using B = MrtBasis<L>;
    constexpr int Q = L::Q;
    SFor<0, Q>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        R ga = g[a];
        SFor<L::D + 1, Q>::run([&](auto R_) {
            constexpr int r = decltype(R_)::value;
            constexpr int m = B::M[r][a];
            if constexpr (B::kind[r] != 2) {
                if constexpr (m == 1)
                    ga = o_add(ga, ck[r]);
                else if constexpr (m == -1)
                    ga = o_sub(ga, ck[r]);
                else if constexpr (m != 0)
                    ga = o_fma(R(m), ck[r], ga);
            }
        });
        g[a] = ga;
    });
}

template <class L, class R, int MODEL, bool FORCE>
__device__ __forceinline__ void collide(R (&g)[L::Q], const R (&F)[3], const Coef<R> &c,
                                        R (&u)[3], R &s_out, R &rho_out)
{
    constexpr bool COMP = MODEL == M_COMP;
    constexpr int H = L::Q / 2;
    R sp[H], sm[H];
    SFor<0, H>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        sp[a] = o_add(g[a], g[opp<L>(a)]);
        sm[a] = o_sub(g[a], g[opp<L>(a)]);
    });
    R s = g[H];
    R j[3] = {R(0), R(0), R(0)};
    SFor<0, H>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        s = o_add(s, sp[a]);
        SFor<0, 3>::run([&](auto K_) {
            constexpr int k = decltype(K_)::value;
            if constexpr (L::e(a, k) == 1)
                j[k] = o_add(j[k], sm[a]);
            else if constexpr (L::e(a, k) == -1)
                j[k] = o_sub(j[k], sm[a]);
        });
    });
    R rho, ir;
    if constexpr (COMP) {
        rho = o_add(s, c.sigma);
        ir = R(1) / rho;
    } else {
        rho = c.rho0;
        ir = c.inv_rho0;
    }
    s_out = s;
    rho_out = rho;
    R jf[3];  // j + F/2 = rho u
    SFor<0, 3>::run([&](auto K_) {
        constexpr int k = decltype(K_)::value;
        if constexpr (FORCE)
            jf[k] = o_fma(R(0.5), F[k], j[k]);
        else
            jf[k] = j[k];
        u[k] = o_mul(jf[k], ir);
    });
    R ck[L::Q];  // MRT: corrections to the BGK update (from the pre-collision g)
    (void)ck;
    if constexpr (MODEL == M_MRT)
        mrt_corrections<L, R, FORCE>(g, F, c, s, rho, ir, jf, u, ck);
    const R uu = o_fma(u[2], u[2], o_fma(u[1], u[1], o_mul(u[0], u[0])));
    R A = o_fma(o_mul(R(-1.5), rho), uu, s);
    if constexpr (FORCE) {
        const R uF = o_fma(u[2], F[2], o_fma(u[1], F[1], o_mul(u[0], F[0])));
        A = o_fma(o_mul(R(-3), c.kf), uF, A);
    }
    const R r3 = o_mul(R(3), rho), r45 = o_mul(R(4.5), rho);
    const R om = c.omega;
    // equilibrium (+ folded source) of pair a: symmetric and antisymmetric
    // parts, feq_a = t (sym + asym), feq_b = t (sym - asym)
    auto pair_eq = [&](auto A_, R &sym, R &asym) {
        constexpr int a = decltype(A_)::value;
        // e.u = (e.j') ir with j' = j (+ F/2): sums first, one product last
        R ej = R(0), eF = R(0);
        (void)eF;
        SFor<0, 3>::run([&](auto K_) {
            constexpr int k = decltype(K_)::value;
            if constexpr (L::e(a, k) == 1) {
                ej = o_add(ej, jf[k]);
                if constexpr (FORCE)
                    eF = o_add(eF, F[k]);
            } else if constexpr (L::e(a, k) == -1) {
                ej = o_sub(ej, jf[k]);
                if constexpr (FORCE)
                    eF = o_sub(eF, F[k]);
            }
        });
        const R eu = o_mul(ej, ir);
        sym = o_fma(o_mul(r45, eu), eu, A);
        asym = o_mul(r3, eu);
        if constexpr (FORCE) {
            sym = o_fma(o_mul(o_mul(R(9), c.kf), eu), eF, sym);
            asym = o_fma(o_mul(R(3), MODEL == M_TRT ? c.kf_m : c.kf), eF, asym);
        }
    };
    if constexpr (MODEL == M_TRT) {
        // Two relaxation times: the even half gp = (g_a + g_b)/2 relaxes at
        // omega towards t sym, the odd half gm = (g_a - g_b)/2 at omega_m
        // towards t asym (the source's odd part carries (1 - omega_m/2));
        // then g_a = gp + gm, g_b = gp - gm.  Built from the pair sums sp, sm
        // of the moment pass, so g itself is dead by now.
        const R omm = c.omega_m;
        SFor<0, H>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            constexpr int b = opp<L>(a);
            const R t = R(L::w(a));
            R sym, asym;
            pair_eq(A_, sym, asym);
            const R hp = o_mul(sp[a], R(0.5)), hm = o_mul(sm[a], R(0.5));
            const R gp = o_fma(om, o_fma(sym, t, -hp), hp);
            // odd part: omm (asym t - hm) + hm; in FP32 the weight's lo part is
            // added to the small difference asym t_hi - hm, where it is not lost
            R gm;
            if constexpr (std::is_same<R, float>::value)
                gm = o_fma(omm, o_fma(asym, w_lo<L>(a), o_fma(asym, w_hi<L>(a), -hm)), hm);
            else
                gm = o_fma(omm, o_fma(asym, t, -hm), hm);
            g[a] = o_add(gp, gm);
            g[b] = o_sub(gp, gm);
        });
    } else {
        SFor<0, H>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            constexpr int b = opp<L>(a);
            const R t = R(L::w(a));
            R sym, asym;
            pair_eq(A_, sym, asym);
            // no product feeds an add directly: each multiply-add is one
            // explicit fma, so no compiler can fuse (and re-round) it
            // differently
            const R at = wmul<L, a>(asym);
            const R fa = o_fma(sym, t, at), fb = o_fma(sym, t, -at);
            g[a] = o_fma(om, o_sub(fa, g[a]), g[a]);
            g[b] = o_fma(om, o_sub(fb, g[b]), g[b]);
        });
    }
    {
        const R t0 = R(L::w(H));
        g[H] = o_fma(om, o_fma(t0, A, -g[H]), g[H]);
    }
    if constexpr (MODEL == M_MRT)
        mrt_apply<L, R>(g, ck);
}

// ---- neighbours -------------------------------------------------------------
// For one axis at coordinate c: node offsets of the upstream node along -e
// for e = +1 (upstream c-1, `op`) and e = -1 (upstream c+1, `om`), and
// whether that upstream node lies beyond a wall.
struct AxisNbr {
    int op, om;
    bool wp, wm;
};

__device__ __forceinline__ AxisNbr axis_general(int c, int n, int stride, bool periodic)
{
    AxisNbr a;
    a.wp = false;
    a.wm = false;
    if (c > 0) {
        a.op = -stride;
    } else {
        a.op = periodic ? (n - 1) * stride : 0;
        a.wp = !periodic;
    }
    if (c < n - 1) {
        a.om = stride;
    } else {
        a.om = periodic ? -(n - 1) * stride : 0;
        a.wm = !periodic;
    }
    return a;
}

__device__ __forceinline__ AxisNbr axis_interior(int stride)
{
    AxisNbr a;
    a.op = -stride;
    a.om = stride;
    a.wp = false;
    a.wm = false;
    return a;
}

// Upstream offset and wall flag of direction a (pull source x - e_a).
template <class L, int a>
__device__ __forceinline__ void upstream(const AxisNbr &X, const AxisNbr &Y, const AxisNbr &Z,
                                         int &off, bool &wall)
{
    constexpr int ex = L::e(a, 0), ey = L::e(a, 1), ez = L::e(a, 2);
    off = 0;
    wall = false;
    if constexpr (ex == 1) {
        off += X.op;
        wall = wall || X.wp;
    } else if constexpr (ex == -1) {
        off += X.om;
        wall = wall || X.wm;
    }
    if constexpr (ey == 1) {
        off += Y.op;
        wall = wall || Y.wp;
    } else if constexpr (ey == -1) {
        off += Y.om;
        wall = wall || Y.wm;
    }
    if constexpr (ez == 1) {
        off += Z.op;
        wall = wall || Z.wp;
    } else if constexpr (ez == -1) {
        off += Z.om;
        wall = wall || Z.wm;
    }
}

template <class L, bool INTERIOR>
__device__ __forceinline__ void make_axes(const StepParams &p, int x, int y, int z, AxisNbr &X,
                                          AxisNbr &Y, AxisNbr &Z)
{
    X = axis_general(x, p.nx, 1, p.periodic & 1);
    if constexpr (INTERIOR) {
        Y = axis_interior(p.nx);
        Z = axis_interior(p.nx * p.ny);
    } else {
        Y = axis_general(y, p.ny, p.nx, p.periodic & 2);
        if constexpr (L::D == 3)
            Z = axis_general(z, p.nz, p.nx * p.ny, p.periodic & 4);
        else
            Z = axis_interior(0);
    }
}

// ---- monitor values of one node (Sec. 3.4 Monitor) ---------------------------
// sum P (shifted: sum g), momentum rho u, kinetic energy rho |u|^2 / 2, |u|^2.
template <class R>
__device__ __forceinline__ void monitor_values(R s, R rho, const R (&u)[3], R (&mon)[6])
{
    const R uu = o_fma(u[2], u[2], o_fma(u[1], u[1], o_mul(u[0], u[0])));
    mon[0] = s;
    mon[1] = o_mul(rho, u[0]);
    mon[2] = o_mul(rho, u[1]);
    mon[3] = o_mul(rho, u[2]);
    mon[4] = o_mul(o_mul(R(0.5), rho), uu);
    mon[5] = uu;
}

template <class R>
__device__ __forceinline__ R warp_sum(R v);
template <class R>
__device__ __forceinline__ R warp_max(R v);

// Block-wide monitor sums of the launch's nodes, written to
// partials[block * kPartialStride + k] in FP64.  Each thread stores its six
// values in shared memory (column k, row threadIdx.x); after a barrier, warp
// w reduces the values k = w, w + nwarps, ... of the whole block in the
// kernel's arithmetic (each lane its threads lane, lane + 32, ... in order,
// then the warp tree; the maximum for k = 5), in a fixed order.  One store per
// value and thread instead of a warp reduction per value and node: at 256^3
// the monitor-fused AA local half went from 385.9 to 378.0 us.  (The gather
// half keeps its own warp sums before the push stores: in this form it was
// slower, 432.7 against 425.0 us.)  Every thread of the block must call it.
template <class R>
__device__ __forceinline__ void block_monitor(const R (&mon)[6], double *partials, size_t b)
{
    __shared__ R col[6 * kMonSlots];
    for (int k = 0; k < 6; ++k)
        col[k * kMonSlots + threadIdx.x] = mon[k];
    __syncthreads();
    const int lane = threadIdx.x & 31, nt = blockDim.x, nwarps = (nt + 31) >> 5;
    for (int k = threadIdx.x >> 5; k < 6; k += nwarps) {
        const R *c = col + k * kMonSlots;
        R v = lane < nt ? c[lane] : R(0);
        if (k == 5) {
            for (int i = lane + 32; i < nt; i += 32)
                v = max(v, c[i]);
            v = warp_max(v);
        } else {
            for (int i = lane + 32; i < nt; i += 32)
                v = o_add(v, c[i]);
            v = warp_sum(v);
        }
        if (lane == 0)
            partials[b * kPartialStride + k] = double(v);
    }
}

// ---- one node of one time step ----------------------------------------------
// INTERIOR: the node's row has neighbours inside the box in y and z (no wall,
// no wrap), so only the x axis needs per-thread boundary logic.
// EARLY_RED (with RED): reduce the monitor values across the warp right after
// the collision and park the warp's sums in wsh[warp], so that they are not
// held in registers through the stores (the AA gather half's push stores
// otherwise take the kernel from 48 to 75 registers); every lane must then
// run the node, idle lanes (active = false) on a copy of a real node, storing
// nothing.
template <class L, int S, int PAT, int MODEL, bool FORCE, bool UOUT, bool INTERIOR,
          bool RED = false, bool EARLY_RED = false>
__device__ __forceinline__ void step_node(const typename Sto<S>::T *src, typename Sto<S>::T *dst,
                                          const StepParams &p, int x, int y, int z,
                                          typename Sto<S>::R (&mon)[6], bool active = true,
                                          double (*wsh)[6] = nullptr)
{
    using T = typename Sto<S>::T;
    using R = typename Sto<S>::R;
    constexpr int Q = L::Q;
    const Coef<R> &c = coef<R>(p);
    const size_t N = (size_t)p.N;
    const int n = x + p.nx * (y + p.ny * z);
    AxisNbr X, Y, Z;
    make_axes<L, INTERIOR>(p, x, y, z, X, Y, Z);
    const bool lid_row = !INTERIOR && p.lid_on && (y == p.ny - 1);

    R g[Q];
    if constexpr (PAT == PAT_LOCAL) {
        // Slot a of x holds the population entering x along e_a; on the top
        // row every e_y = -1 population has crossed the moving wall, and its
        // lid term is added here, at read time, exactly as the pull scheme
        // does, so that both schemes round identically.
        const bool top = p.lid_on && (y == p.ny - 1);
        SFor<0, Q>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            R v = Sto<S>::dec(ld(src + a * N + n));
            if constexpr (L::e(a, 1) == -1) {
                if (top)
                    v += c.lid[a];
            }
            g[a] = v;
        });
    } else {
        SFor<0, Q>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            constexpr int b = opp<L>(a);
            const T *ptr;
            if constexpr (INTERIOR) {
                // only x can wrap or meet a wall; y and z shifts are the
                // uniform row offsets
                constexpr int ex = L::e(a, 0);
                const long long o = PAT == PAT_PULL ? p.pull_off[a] : p.push_off[b];
                const T *s0 = src + n;
                if constexpr (ex == 0) {
                    ptr = s0 + o;
                } else {
                    const bool wall = ex == 1 ? X.wp : X.wm;
                    const int xo = ex == 1 ? X.op : X.om;
                    ptr = wall ? s0 + (size_t)(PAT == PAT_PULL ? b : a) * N : (s0 + xo) + o;
                }
            } else {
                int off;
                bool wall;
                upstream<L, a>(X, Y, Z, off, wall);
                if constexpr (PAT == PAT_PULL)
                    ptr = wall ? src + b * N + n : src + a * N + (n + off);
                else
                    ptr = wall ? src + a * N + n : src + b * N + (n + off);
            }
            R v;
            if constexpr (EARLY_RED)  // an idle lane reads nothing (the slots are owned)
                v = active ? Sto<S>::dec(ld(ptr)) : R(0);
            else
                v = Sto<S>::dec(ld(ptr));
            if constexpr (L::e(a, 1) == -1) {
                if (lid_row)
                    v += c.lid[a];
            }
            g[a] = v;
        });
    }
    R F[3] = {R(0), R(0), R(0)};
    if constexpr (FORCE) {
        SFor<0, L::D>::run([&](auto K_) {
            constexpr int k = decltype(K_)::value;
            F[k] = R(p.F[k * N + n]);
        });
    }
    R u[3], s_, rho_;
    collide<L, R, MODEL, FORCE>(g, F, c, u, s_, rho_);
    if constexpr (RED)
        monitor_values(s_, rho_, u, mon);
    if constexpr (RED && EARLY_RED) {
        R w[6];
        for (int k = 0; k < 5; ++k)
            w[k] = warp_sum(active ? mon[k] : R(0));
        w[5] = warp_max(active ? mon[5] : R(0));
        if ((threadIdx.x & 31) == 0)
            for (int k = 0; k < 6; ++k)
                wsh[threadIdx.x >> 5][k] = double(w[k]);
        if (!active)
            return;
    }
    if constexpr (UOUT) {
        SFor<0, L::D>::run([&](auto K_) {
            constexpr int k = decltype(K_)::value;
            ((R *)p.u_out)[k * N + n] = u[k];
        });
    }
    SFor<0, Q>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        constexpr int b = opp<L>(a);
        if constexpr (PAT == PAT_PULL) {
            st(dst + a * N + n, Sto<S>::enc(g[a]));
        } else if constexpr (PAT == PAT_LOCAL) {
            st(dst + b * N + n, Sto<S>::enc(g[a]));
        } else {
            // push f*_a to x + e_a, whose upstream along -e_b is x
            if constexpr (INTERIOR) {
                constexpr int ex = L::e(a, 0);
                T *d0 = dst + n;
                if constexpr (ex == 0) {
                    st(d0 + p.push_st[a], Sto<S>::enc(g[a]));
                } else {
                    const bool wall = ex == 1 ? X.wm : X.wp;
                    const int xo = ex == 1 ? X.om : X.op;
                    st(wall ? d0 + (size_t)b * N : (d0 + xo) + p.push_st[a], Sto<S>::enc(g[a]));
                }
                return;
            }
            int off;
            bool wall;
            upstream<L, b>(X, Y, Z, off, wall);
            if (wall) {
                // bounced: stays at x as the population entering along e_b
                // (its lid term, if any, is added when it is read)
                st(dst + b * N + n, Sto<S>::enc(g[a]));
            } else {
                st(dst + a * N + (n + off), Sto<S>::enc(g[a]));
            }
        }
    });
}

// grid: (ceil(nx/blockDim.x), ny, nz); one node per thread.
template <class L, int S, int PAT, int MODEL, bool FORCE, bool UOUT, bool RED>
__device__ __forceinline__ void step_kernel_body(const typename Sto<S>::T *src,
                                                 typename Sto<S>::T *dst, const StepParams &p,
                                                 int bx, int y, int z, size_t bid)
{
    using R = typename Sto<S>::R;
    const int x = bx * blockDim.x + threadIdx.x;
    if constexpr (!RED) {  // no block-wide step follows: idle threads may leave
        if (x >= p.nx)
            return;
    }
    R mon[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    if constexpr (RED && PAT == PAT_GATHER) {
        // warp sums before the stores (see EARLY_RED); idle lanes recompute
        // the row's last node
        __shared__ double wsh[8][6];
        const bool active = x < p.nx;
        const int xc = active ? x : p.nx - 1;
        const bool interior = y > 0 && y < p.ny - 1 && (L::D == 2 || (z > 0 && z < p.nz - 1));
        if (interior)
            step_node<L, S, PAT, MODEL, FORCE, UOUT, true, true, true>(src, dst, p, xc, y, z, mon,
                                                                       active, wsh);
        else
            step_node<L, S, PAT, MODEL, FORCE, UOUT, false, true, true>(src, dst, p, xc, y, z, mon,
                                                                        active, wsh);
        __syncthreads();
        if (threadIdx.x < 6) {
            const int k = threadIdx.x, nw = (blockDim.x + 31) >> 5;
            double r = wsh[0][k];
            for (int i = 1; i < nw; ++i)
                r = (k == 5) ? fmax(r, wsh[i][k]) : r + wsh[i][k];
            p.partials[bid * kPartialStride + k] = r;
        }
        return;
    }
    if (x < p.nx) {
        if constexpr (PAT == PAT_LOCAL) {
            step_node<L, S, PAT, MODEL, FORCE, UOUT, true, RED>(src, dst, p, x, y, z, mon);
        } else {
            const bool interior =
                y > 0 && y < p.ny - 1 && (L::D == 2 || (z > 0 && z < p.nz - 1));
            if (interior)
                step_node<L, S, PAT, MODEL, FORCE, UOUT, true, RED>(src, dst, p, x, y, z, mon);
            else
                step_node<L, S, PAT, MODEL, FORCE, UOUT, false, RED>(src, dst, p, x, y, z, mon);
        }
    }
    if constexpr (RED)
        block_monitor(mon, p.partials, bid);
}

__device__ __forceinline__ size_t grid_block_index()
{
    return blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
}

// (__launch_bounds__ with an explicit minimum of 1 block lets nvcc roughly
// double the register count of these kernels and halves their occupancy;
// the thread bound alone keeps them at 40-48 registers.)
template <class L, int S, int PAT, int MODEL, bool FORCE, bool UOUT, bool RED = false>
__global__ void __launch_bounds__(256) k_step(const typename Sto<S>::T *src,
                                              typename Sto<S>::T *dst, const StepParams p)
{
    step_kernel_body<L, S, PAT, MODEL, FORCE, UOUT, RED>(src, dst, p, blockIdx.x, blockIdx.y,
                                                         blockIdx.z, grid_block_index());
}

// The step held to MINB blocks per SM (D3Q27 with 16-bit storage: the
// compiler's 70-72 registers leave three blocks per SM to these
// latency-bound kernels).
template <class L, int S, int PAT, int MODEL, bool FORCE, int MINB>
__global__ void __launch_bounds__(256, MINB) k_step_bounded(const typename Sto<S>::T *src,
                                                            typename Sto<S>::T *dst,
                                                            const StepParams p)
{
    step_kernel_body<L, S, PAT, MODEL, FORCE, false, false>(src, dst, p, blockIdx.x, blockIdx.y,
                                                            blockIdx.z, grid_block_index());
}

// The AA gather half with the monitor fused in: held to five blocks per SM
// (48 registers, a few bytes spilled) instead of the 62 it takes unbounded;
// D3Q19 FP32 without force to six (40 registers; measured at 512^3: 3.41 ms
// at six, 3.68 at five, 3.86 at four, 4.42 at seven).  FP64 (three) and
// D3Q27 (four) get more registers: at five they spill 100-1200 bytes.
template <class L, int S, bool FORCE>
constexpr int kGatherRedMinBlocks = S == ST_F64                          ? 3
                                    : L::Q == 27                         ? 4
                                    : (L::Q == 19 && S == ST_F32 && !FORCE) ? 6
                                                                         : 5;
template <class L, int S, int MODEL, bool FORCE>
__global__ void __launch_bounds__(256, (kGatherRedMinBlocks<L, S, FORCE>)) k_step_gather_red(const typename Sto<S>::T *src,
                                                            typename Sto<S>::T *dst,
                                                            const StepParams p)
{
    step_kernel_body<L, S, PAT_GATHER, MODEL, FORCE, false, true>(
        src, dst, p, blockIdx.x, blockIdx.y, blockIdx.z, grid_block_index());
}

// A node the plain kernel cannot update in a box with per-face boundaries or
// obstacles: solid, with an obstacle link, or on an inlet, outflow, symmetry
// or nodal face.
__device__ __forceinline__ bool needs_general(const StepParams &p, int n, int x, int y, int z)
{
    const int f = p.open_faces;
    bool open = ((f & 1) && x < p.xm) || ((f & 2) && x >= p.nx - p.xm) || ((f & 4) && y == 0) ||
                ((f & 8) && y == p.ny - 1) || ((f & 16) && z == 0) || ((f & 32) && z == p.nz - 1);
    return open || (p.links && p.links[n] != 0u);
}

// The pull step of a box with per-face boundaries or obstacles on every node
// the plain kernel can update (walls, lid and periodic faces only, no
// obstacle link), which it computes exactly as the general kernel does; the
// other nodes are left to the general kernel's node-list launch.  MON: 0,
// 1 = monitor sums of these nodes, 2 = obstacle force (zero here).
template <class L, int S, int MODEL, bool FORCE, int MON>
__global__ void __launch_bounds__(256) k_step_skip(const typename Sto<S>::T *src,
                                                   typename Sto<S>::T *dst, const StepParams p)
{
    using R = typename Sto<S>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    const int n = x + p.nx * (y + p.ny * z);
    const bool active = x < p.nx && !needs_general(p, n, x, y, z);
    if constexpr (MON == 2) {
        if (threadIdx.x < kReduceVals)
            p.partials[grid_block_index() * kPartialStride + threadIdx.x] = 0.0;
    }
    if constexpr (MON != 1) {
        if (!active)
            return;
    }
    R mon[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    if (active) {
        const bool interior = y > 0 && y < p.ny - 1 && (L::D == 2 || (z > 0 && z < p.nz - 1));
        if (interior)
            step_node<L, S, PAT_PULL, MODEL, FORCE, false, true, MON == 1>(src, dst, p, x, y, z, mon);
        else
            step_node<L, S, PAT_PULL, MODEL, FORCE, false, false, MON == 1>(src, dst, p, x, y, z,
                                                                            mon);
    }
    if constexpr (MON == 1)
        block_monitor(mon, p.partials, grid_block_index());
}

// ---- initialisation (Sec. 2.2: f = feq(p, u), then the first collision) -----
// p0: N values or NULL (p = 1/3); u0: d*N values or NULL (u = 0); IN is
// their type (FP64, or FP32 for lbm_init_f32).

template <class L, int S, bool AA, int MODEL, bool FORCE, class IN>
__global__ void __launch_bounds__(256) k_init(typename Sto<S>::T *dst, const StepParams p,
                                              const IN *p0, const IN *u0)
{
    constexpr int Q = L::Q;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.nx)
        return;
    using R = typename Sto<S>::R;
    const size_t N = (size_t)p.N;
    const int n = x + p.nx * (y + p.ny * z);
    const Coef<R> &c = coef<R>(p);
    // shifted pressure P - sigma taken in FP64 before rounding to R
    const double P = p0 ? 3.0 * double(p0[n]) : 1.0;
    const R dP = R(P - double(c.sigma));
    R u[3] = {R(0), R(0), R(0)};
    if (u0)
        for (int k = 0; k < L::D; ++k)
            u[k] = R(u0[k * N + n]);
    const R uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const R rho = MODEL == M_COMP ? R(P) : c.rho0;
    R g[Q];
    SFor<0, Q>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        const R t = R(L::w(a));
        const R eu = R(L::e(a, 0)) * u[0] + R(L::e(a, 1)) * u[1] + R(L::e(a, 2)) * u[2];
        const R poly = R(3) * eu + R(4.5) * eu * eu - R(1.5) * uu;
        // feq - sigma t = t [(P - sigma) + rho poly]  (Eq. (incompressible_feq) / Eq. (feq))
        g[a] = t * (dP + rho * poly);
    });
    if constexpr (FORCE) {
        R F[3] = {R(0), R(0), R(0)};
        for (int k = 0; k < L::D; ++k)
            F[k] = R(p.F[k * N + n]);
        R uc[3], s_, rho_;
        collide<L, R, MODEL, true>(g, F, c, uc, s_, rho_);
    }
    SFor<0, Q>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        const int slot = AA ? opp<L>(a) : a;
        dst[slot * N + n] = Sto<S>::enc(g[a]);
    });
}

// ---- moments + FP64 reduction (Sec. 3.4 PostProcessing and Monitor) ---------
struct MomParams {
    void *p_out;  // N values or NULL
    void *u_out;  // d*N values or NULL
    int out_f32;
    double *partials;  // gridDim.x * kPartialStride doubles, or NULL
    int nseg;          // x-segments * ny * nz
    int xseg;          // x-segments per row
    const unsigned *links;  // per-node link words: solid nodes report zero
};

template <class R>
__device__ __forceinline__ R warp_sum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <class R>
__device__ __forceinline__ R warp_max(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Moments of one node from its populations g (in the storage's shift): s =
// sum g (the shifted pressure sum), rho, and u = (j* - F/2)/rho from the
// post-collision momentum j* = j + F.  Shared by every kernel that reduces or
// outputs the moments of a state, so that they agree bit for bit.
template <class L, class R, bool COMP, bool FORCE>
__device__ __forceinline__ void moments_of(const R (&g)[L::Q], const StepParams &p, int n, R &s,
                                           R &rho, R (&u)[3])
{
    constexpr int Q = L::Q;
    const Coef<R> &c = coef<R>(p);
    const size_t N = (size_t)p.N;
    R j[3] = {R(0), R(0), R(0)};
    s = R(0);
    SFor<0, Q>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        s = o_add(s, g[a]);
        SFor<0, 3>::run([&](auto K_) {
            constexpr int k = decltype(K_)::value;
            if constexpr (L::e(a, k) == 1)
                j[k] = o_add(j[k], g[a]);
            else if constexpr (L::e(a, k) == -1)
                j[k] = o_sub(j[k], g[a]);
        });
    });
    rho = COMP ? o_add(s, c.sigma) : c.rho0;
    const R ir = COMP ? R(1) / rho : c.inv_rho0;
    for (int k = 0; k < 3; ++k) {
        R jk = j[k];
        if constexpr (FORCE) {
            if (k < L::D)
                jk = o_fma(R(-0.5), R(p.F[k * N + n]), jk);
        }
        u[k] = o_mul(jk, ir);
    }
}

// Node n's moments from a stored state in form FORM (moments_of on the
// populations entering the node).
template <class L, int S, int FORM, bool COMP, bool FORCE>
__device__ __forceinline__ void node_moments(const typename Sto<S>::T *src, const StepParams &p,
                                             int x, int y, int z, int n,
                                             typename Sto<S>::R &s, typename Sto<S>::R &rho,
                                             typename Sto<S>::R (&u)[3])
{
    using R = typename Sto<S>::R;
    constexpr int Q = L::Q;
    const size_t N = (size_t)p.N;
    R g[Q];
    if constexpr (FORM == FORM_LOCAL) {
        SFor<0, Q>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            g[a] = Sto<S>::dec(src[a * N + n]);
        });
    } else if constexpr (FORM == FORM_SWAPPED) {
        SFor<0, Q>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            g[a] = Sto<S>::dec(src[opp<L>(a) * N + n]);
        });
    } else {
        AxisNbr X, Y, Z;
        make_axes<L, false>(p, x, y, z, X, Y, Z);
        SFor<0, Q>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            constexpr int b = opp<L>(a);
            int off;
            bool wall;
            upstream<L, b>(X, Y, Z, off, wall);
            if (wall) {
                g[a] = Sto<S>::dec(src[b * N + n]);
            } else {
                g[a] = Sto<S>::dec(src[a * N + (n + off)]);
            }
        });
    }
    moments_of<L, R, COMP, FORCE>(g, p, n, s, rho, u);
}

// Grid-stride over x-segments of rows; each block keeps FP64 partial sums of
// the per-node values (reduced across a warp in the kernel's arithmetic
// first) and writes them to partials[blockIdx.x].
template <class L, int S, int FORM, bool COMP, bool FORCE>
__global__ void __launch_bounds__(256) k_moments(const typename Sto<S>::T *src, const StepParams p,
                                                 const MomParams m)
{
    using R = typename Sto<S>::R;
    const Coef<R> &c = coef<R>(p);
    const size_t N = (size_t)p.N;
    // lane k < 5 keeps the FP64 running sum of monitor value k: one FP64 add
    // per warp and segment instead of five (B300's FP64 rate is a small
    // fraction of FP32); the maximum stays in the kernel's arithmetic, where
    // it is exact
    double acc = 0.0;
    R accmax = R(0);
    const int lane = threadIdx.x & 31;
    for (int seg = blockIdx.x; seg < m.nseg; seg += gridDim.x) {
        const int xs = seg % m.xseg;
        const int row = seg / m.xseg;
        const int y = row % p.ny, z = row / p.ny;
        const int x = xs * blockDim.x + threadIdx.x;
        R vals[kReduceVals] = {R(0), R(0), R(0), R(0), R(0), R(0)};
        const int n0 = x + p.nx * (y + p.ny * z);
        const bool solid = x < p.nx && m.links && (m.links[n0] >> 31);
        if (solid) {
            if (m.p_out) {
                if (m.out_f32)
                    ((float *)m.p_out)[n0] = 0.f;
                else
                    ((double *)m.p_out)[n0] = 0.0;
            }
            if (m.u_out) {
                for (int k = 0; k < L::D; ++k) {
                    if (m.out_f32)
                        ((float *)m.u_out)[k * N + n0] = 0.f;
                    else
                        ((double *)m.u_out)[k * N + n0] = 0.0;
                }
            }
        }
        if (x < p.nx && !solid) {
            const int n = n0;
            R s_, rho, u[3];
            node_moments<L, S, FORM, COMP, FORCE>(src, p, x, y, z, n, s_, rho, u);
            if (m.p_out) {
                const R pv = (s_ + c.sigma) * R(1.0 / 3.0);
                if (m.out_f32)
                    ((float *)m.p_out)[n] = float(pv);
                else
                    ((double *)m.p_out)[n] = double(pv);
            }
            if (m.u_out) {
                for (int k = 0; k < L::D; ++k) {
                    if (m.out_f32)
                        ((float *)m.u_out)[k * N + n] = float(u[k]);
                    else
                        ((double *)m.u_out)[k * N + n] = double(u[k]);
                }
            }
            monitor_values(s_, rho, u, vals);
        }
        if (m.partials) {
            R mine = R(0);
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const R w = warp_sum(vals[k]);
                mine = lane == k ? w : mine;
            }
            if (lane < 5)
                acc += double(mine);
            accmax = max(accmax, warp_max(vals[5]));
        }
    }
    if (!m.partials)
        return;
    __shared__ double sh[8][kReduceVals];
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (lane < 5)
        sh[warp][lane] = acc;
    else if (lane == 5)
        sh[warp][5] = double(accmax);
    __syncthreads();
    if (threadIdx.x < kReduceVals) {
        const int k = threadIdx.x;
        double r = sh[0][k];
        for (int w = 1; w < nwarps; ++w)
            r = (k == 5) ? fmax(r, sh[w][k]) : r + sh[w][k];
        m.partials[blockIdx.x * kPartialStride + k] = r;
    }
}

// One block: fixed-order sum of the per-block partials into out[0..5].
static __global__ void __launch_bounds__(256) k_reduce_finish(const double *partials, int nblocks,
                                                       double *out)
{
    __shared__ double sh[256][kReduceVals];
    double acc[kReduceVals] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < kReduceVals; ++k)
            acc[k] = (k == 5) ? fmax(acc[k], partials[b * kPartialStride + k])
                              : acc[k] + partials[b * kPartialStride + k];
    for (int k = 0; k < kReduceVals; ++k)
        sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < kReduceVals; ++k)
                sh[threadIdx.x][k] = (k == 5) ? fmax(sh[threadIdx.x][k], sh[threadIdx.x + s][k])
                                              : sh[threadIdx.x][k] + sh[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x < kReduceVals)
        out[threadIdx.x] = sh[0][threadIdx.x];
}

// First stage of the fused monitor: block b sums partials [b*chunk, (b+1)*chunk)
// of the step kernel's blocks, in order, into out[b].
static __global__ void __launch_bounds__(256) k_reduce_chunks(const double *in, long long nin,
                                                              long long chunk, double *out)
{
    __shared__ double sh[256][kReduceVals];
    double acc[kReduceVals] = {0, 0, 0, 0, 0, 0};
    const long long lo = blockIdx.x * chunk;
    const long long hi = lo + chunk < nin ? lo + chunk : nin;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x)
        for (int k = 0; k < kReduceVals; ++k)
            acc[k] = (k == 5) ? fmax(acc[k], in[i * kPartialStride + k])
                              : acc[k] + in[i * kPartialStride + k];
    for (int k = 0; k < kReduceVals; ++k)
        sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < kReduceVals; ++k)
                sh[threadIdx.x][k] = (k == 5) ? fmax(sh[threadIdx.x][k], sh[threadIdx.x + s][k])
                                              : sh[threadIdx.x][k] + sh[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x < kReduceVals)
        out[blockIdx.x * kPartialStride + threadIdx.x] = sh[0][threadIdx.x];
}

// ---- adjoint parameters (kernels in lbm_adjoint.cuh) -------------------------
struct AdjParams {
    const void *lam_in;   // lambda^{k+1}, Q*N (R)
    void *lam_out;        // lambda^k, Q*N (R)
    const void *u_k;      // u^k, d*N (R)
    void *gF;             // per-segment force gradient, d*N (R), accumulated
    double *gU_part;      // per top-row block: 4 doubles, accumulated over steps
    const void *state;    // seed: final post-collision state (pull-scheme layout)
    double *dJdF;         // segment flush: FP64 total, d*N
    int xseg;
};

// ---- host-side launch descriptors ----------------------------------------------
enum Kind {
    K_STEP = 0,
    K_INIT = 1,
    K_MOMENTS = 2,
    K_ADJ = 3,
    K_SEED = 4,
    K_FLUSH = 5,
    K_LINKS = 6,
    K_FLAGS = 7
};

struct Launch {
    int kind;
    int storage;
    int pattern;  // K_STEP: Pattern; K_MOMENTS: Form; K_INIT: 1 = AA slots
    bool comp, force, uout;
    int model;  // K_STEP / K_INIT: Model
    const void *src;
    void *dst;
    StepParams sp;
    const void *p0, *u0;
    bool in_f32;  // K_INIT: p0 / u0 are FP32 (else FP64)
    MomParams mp;
    AdjParams ap;
    size_t count;  // K_FLUSH
    bool pair;     // K_STEP: two nodes per thread, 32-bit accesses (lbm_pair.cuh)
    bool geo;      // K_STEP: the general kernel (per-face boundaries, obstacles; lbm_geo.cuh)
    bool skip;     // K_STEP: the plain pull kernel on the nodes it can update (k_step_skip)
    int mon;       // K_STEP with geo or skip: 0, 1 = monitor sums, 2 = obstacle force sums
    unsigned char *flags;        // K_FLAGS: one byte per node
    const unsigned char *solid;  // K_LINKS: N bytes, nonzero = solid
    unsigned *links;             // K_LINKS: output link words
    unsigned long long *nsolid;  // K_LINKS: number of solid nodes (added to)
    dim3 grid, block;
    cudaStream_t stream;
};

// Per-lattice entry points (one translation unit each).
cudaError_t launch_d2q9(const Launch &l);
cudaError_t launch_d3q19(const Launch &l);
cudaError_t launch_d3q27(const Launch &l);
cudaError_t launch_finish(const double *partials, int nblocks, double *out, cudaStream_t s);
cudaError_t launch_chunks(const double *in, long long nin, double *out, int nout, cudaStream_t s);

}  // namespace lbm
