// lbm_geo.cuh -- the general step kernel: per-face boundary conditions and
// solid obstacles (the workloads of Sec. 4-5: channel flow past a cylinder,
// flow past a sphere).
//
// Pull scheme, one node per thread, the same fused gather -> collide -> store
// as k_step.  The population entering fluid node x along e_a is found by
// moving to x - e_a and fixing every coordinate that leaves the box by the
// face it crosses:
//   periodic   wraps;
//   wall       half-way bounce-back, f_a(x) = f*_abar(x), plus the lid term
//              2 t_a rho0 (e_a . U)/c_s^2 on the +y wall;
//   inlet      half-way bounce-back with the term of the inlet velocity at x
//              (wins over the lid on a link crossing both);
//   outflow    pressure outlet by anti-bounce-back,
//              f_a(x) = -f*_abar(x) + 2 feq+_a(P_out, u(x)), feq+ the even
//              half of the equilibrium, u(x) from the node's own
//              post-collision populations;
//   symmetry   the coordinate stays that of x and the direction's component
//              normal to the face is reflected (specular, free slip);
//   nodal      the paper's modified nodal bounce-back (Sec. 2.2, Eq. (bb)):
//              the wall lies on the boundary nodes, which collide like the
//              bulk; f_a(x) = f_abar(x) after propagation, the opposite
//              population that has just arrived from inside (plus the lid
//              term on +y; the node's own f*_abar(x) where that one comes
//              from outside too, as at corners).
// A wall or inlet crossing wins over a nodal one, then outflow, then the
// rest.  If the node so found is solid (bit a of the node's link word),
// the population bounces back at x, and the link's momentum exchange
// 2 f*_abar(x) e_abar counts towards the force on the obstacle (Sec. 5).
// Solid nodes (bit 31) are not updated.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

// lbm_face of include/lbm.h
enum FaceType {
    F_PERIODIC = 0,
    F_WALL = 1,
    F_INLET = 2,
    F_OUTFLOW = 3,
    F_SYMMETRY = 4,
    F_NODAL = 5
};

// What a link crossing one side of one axis does; OR-ed over the components
// of a direction.
enum SideKind : unsigned {
    SK_BOUNCE = 1u,  // wall or inlet: half-way bounce-back
    SK_LID = 2u,     // with the moving lid's term (the +y wall)
    SK_INLET = 4u,   // with the inlet velocity's term
    SK_OUT = 8u,     // pressure outlet
    SK_SYM = 16u,    // symmetry plane
    SK_NODAL = 32u,  // nodal bounce-back (with SK_LID on the +y face)
};
constexpr unsigned kSolidBit = 1u << 31;

struct AxisG {
    int op, om;       // node offsets of the upstream node for e = +1 / e = -1
    unsigned kp, km;  // SideKind of those two links
};

__device__ __forceinline__ unsigned side_kind(int type, bool lid)
{
    switch (type) {
    case F_WALL:
        return SK_BOUNCE | (lid ? SK_LID : 0u);
    case F_INLET:
        return SK_BOUNCE | SK_INLET;
    case F_OUTFLOW:
        return SK_OUT;
    case F_SYMMETRY:
        return SK_SYM;
    case F_NODAL:
        return SK_NODAL | (lid ? SK_LID : 0u);
    default:
        return 0u;
    }
}

// Axis of extent n and node stride `stride` at coordinate c; faces of types
// tlo (coordinate -1 side) and thi (coordinate n side).
__device__ __forceinline__ AxisG axis_faces(int c, int n, int stride, int tlo, int thi,
                                            bool lid_hi)
{
    AxisG a;
    a.kp = 0u;
    a.km = 0u;
    if (c > 0) {
        a.op = -stride;
    } else {
        a.op = tlo == F_PERIODIC ? (n - 1) * stride : 0;
        a.kp = side_kind(tlo, false);
    }
    if (c < n - 1) {
        a.om = stride;
    } else {
        a.om = thi == F_PERIODIC ? -(n - 1) * stride : 0;
        a.km = side_kind(thi, lid_hi);
    }
    return a;
}

__device__ __forceinline__ AxisG axis_open(int stride)
{
    AxisG a;
    a.op = -stride;
    a.om = stride;
    a.kp = 0u;
    a.km = 0u;
    return a;
}

// Link a of the node: offset of its upstream node, the OR of its SideKinds,
// and the slot to read there (a, or its reflection across symmetry faces).
template <class L, int a>
__device__ __forceinline__ void link_of(const AxisG &X, const AxisG &Y, const AxisG &Z, int &off,
                                        unsigned &kind, int &slot)
{
    constexpr int ex = L::e(a, 0), ey = L::e(a, 1), ez = L::e(a, 2);
    const unsigned kx = ex == 1 ? X.kp : ex == -1 ? X.km : 0u;
    const unsigned ky = ey == 1 ? Y.kp : ey == -1 ? Y.km : 0u;
    const unsigned kz = ez == 1 ? Z.kp : ez == -1 ? Z.km : 0u;
    off = (ex == 1 ? X.op : ex == -1 ? X.om : 0) + (ey == 1 ? Y.op : ey == -1 ? Y.om : 0) +
          (ez == 1 ? Z.op : ez == -1 ? Z.om : 0);
    kind = kx | ky | kz;
    slot = a;
    if (kind & SK_SYM)
        slot = L::index_of((kx & SK_SYM) ? -ex : ex, (ky & SK_SYM) ? -ey : ey,
                           (kz & SK_SYM) ? -ez : ez);
}

template <class L>
__device__ __forceinline__ void geo_axes(const StepParams &p, int x, int y, int z, bool interior,
                                         AxisG &X, AxisG &Y, AxisG &Z)
{
    X = axis_faces(x, p.nx, 1, p.face[0], p.face[1], false);
    if (interior) {
        Y = axis_open(p.nx);
        Z = axis_open(p.nx * p.ny);
    } else {
        Y = axis_faces(y, p.ny, p.nx, p.face[2], p.face[3], p.lid_on != 0);
        if constexpr (L::D == 3)
            Z = axis_faces(z, p.nz, p.nx * p.ny, p.face[4], p.face[5], false);
        else
            Z = axis_open(0);
    }
}

// One fluid node of one step.  mon: monitor values (MON == 1); fo: its
// momentum exchange with obstacles (MON == 2).
template <class L, int S, int MODEL, bool FORCE, int MON, bool INTERIOR>
__device__ __forceinline__ void geo_node(const typename Sto<S>::T *src, typename Sto<S>::T *dst,
                                         const StepParams &p, int x, int y, int z,
                                         typename Sto<S>::R (&mon)[6],
                                         typename Sto<S>::R (&fo)[3])
{
    using R = typename Sto<S>::R;
    constexpr int Q = L::Q;
    const Coef<R> &c = coef<R>(p);
    const size_t N = (size_t)p.N;
    const int n = x + p.nx * (y + p.ny * z);
    const unsigned lw = p.links ? p.links[n] : 0u;
    if (lw & kSolidBit)
        return;
    AxisG X, Y, Z;
    geo_axes<L>(p, x, y, z, INTERIOR, X, Y, Z);
    const unsigned any = X.kp | X.km | Y.kp | Y.km | Z.kp | Z.km;

    R F[3] = {R(0), R(0), R(0)};
    if constexpr (FORCE) {
        SFor<0, L::D>::run([&](auto K_) {
            constexpr int k = decltype(K_)::value;
            F[k] = R(p.F[k * N + n]);
        });
    }
    // inlet velocity at this node's place on the inlet face
    R uin[3] = {R(0), R(0), R(0)};
    if ((any & SK_INLET) && p.inlet) {
        const int axis = p.inlet_face >> 1;
        const size_t idx = axis == 0 ? (size_t)y + (size_t)p.ny * z
                           : axis == 1 ? (size_t)x + (size_t)p.nx * z
                                       : (size_t)x + (size_t)p.nx * y;
        const size_t nf = axis == 0 ? (size_t)p.ny * p.nz
                          : axis == 1 ? (size_t)p.nx * p.nz
                                      : (size_t)p.nx * p.ny;
        for (int k = 0; k < L::D; ++k)
            uin[k] = R(p.inlet[k * nf + idx]);
    }
    // outlet node: velocity from its own post-collision populations
    // (collision keeps P and adds F to j: u = (j* - F/2)/rho)
    R ub[3] = {R(0), R(0), R(0)}, ubb = R(0);
    if (any & SK_OUT) {
        R s = R(0), j[3] = {R(0), R(0), R(0)};
        SFor<0, Q>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            const R v = Sto<S>::dec(src[a * N + n]);
            s = o_add(s, v);
            SFor<0, 3>::run([&](auto K_) {
                constexpr int k = decltype(K_)::value;
                if constexpr (L::e(a, k) == 1)
                    j[k] = o_add(j[k], v);
                else if constexpr (L::e(a, k) == -1)
                    j[k] = o_sub(j[k], v);
            });
        });
        const R ir = MODEL == M_COMP ? R(1) / o_add(s, c.sigma) : c.inv_rho0;
        for (int k = 0; k < 3; ++k)
            ub[k] = o_mul(FORCE ? o_fma(R(-0.5), F[k], j[k]) : j[k], ir);
        ubb = o_fma(ub[2], ub[2], o_fma(ub[1], ub[1], o_mul(ub[0], ub[0])));
    }

    // all loads first (straight-line, so every one is in flight before the
    // first value is decoded), then the boundary terms
    using T = typename Sto<S>::T;
    T raw[Q];
    SFor<0, Q>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        constexpr int b = opp<L>(a);
        int off, slot;
        unsigned kind;
        link_of<L, a>(X, Y, Z, off, kind, slot);
        const bool own = (kind & (SK_BOUNCE | SK_OUT | SK_NODAL)) || ((lw >> a) & 1u);
        raw[a] = ld(own ? src + b * N + n : src + (size_t)slot * N + (n + off));
    });
    R g[Q];
    SFor<0, Q>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        constexpr int ex = L::e(a, 0), ey = L::e(a, 1), ez = L::e(a, 2);
        const R t = R(L::w(a));
        int off, slot;
        unsigned kind;
        link_of<L, a>(X, Y, Z, off, kind, slot);
        R v = Sto<S>::dec(raw[a]);
        if (kind & SK_BOUNCE) {
            if (kind & SK_INLET) {
                const R eu = R(ex) * uin[0] + R(ey) * uin[1] + R(ez) * uin[2];
                v = o_fma(o_mul(R(6.0 * L::w(a)), c.rho0), eu, v);
            } else if (kind & SK_LID) {
                v = o_add(v, c.lid[a]);
            }
        } else if (kind & SK_NODAL) {
            // fallback f*_abar(x); replaced below where the opposite
            // population streamed in
        } else if (kind & SK_OUT) {
            const R eu = R(ex) * ub[0] + R(ey) * ub[1] + R(ez) * ub[2];
            const R q = o_fma(o_mul(R(4.5), eu), eu, o_mul(R(-1.5), ubb));
            v = o_fma(t, c.pout2, o_fma(o_mul(R(2.0 * L::w(a)), c.pout_r), q, -v));
        } else if ((lw >> a) & 1u) {
            if constexpr (MON == 2) {
                // f*_b(x) leaves towards the solid and returns reversed
                const R fb2 = o_mul(R(2), o_fma(c.sigma, t, v));
                if constexpr (ex != 0)
                    fo[0] = o_fma(R(-ex), fb2, fo[0]);
                if constexpr (ey != 0)
                    fo[1] = o_fma(R(-ey), fb2, fo[1]);
                if constexpr (ez != 0)
                    fo[2] = o_fma(R(-ez), fb2, fo[2]);
            }
        }
        g[a] = v;
    });
    if (any & SK_NODAL) {
        SFor<0, Q>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            constexpr int b = opp<L>(a);
            int off, slot, offb, slotb;
            unsigned kind, kindb;
            link_of<L, a>(X, Y, Z, off, kind, slot);
            if ((kind & (SK_BOUNCE | SK_NODAL)) != SK_NODAL)
                return;
            link_of<L, b>(X, Y, Z, offb, kindb, slotb);
            const bool streamed =
                !(kindb & (SK_BOUNCE | SK_OUT | SK_NODAL)) && !((lw >> b) & 1u);
            R v = streamed ? g[b] : g[a];
            if (kind & SK_LID)
                v = o_add(v, c.lid[a]);
            g[a] = v;
        });
    }
    R u[3], s_, rho_;
    collide<L, R, MODEL, FORCE>(g, F, c, u, s_, rho_);
    if constexpr (MON == 1)
        monitor_values(s_, rho_, u, mon);
    SFor<0, Q>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        st(dst + a * N + n, Sto<S>::enc(g[a]));
    });
}

// grid: (ceil(nx/blockDim.x), ny, nz); one node per thread.  MON: 0, 1 =
// per-block monitor sums, 2 = per-block obstacle force sums, both into
// p.partials.
template <class L, int S, int MODEL, bool FORCE, int MON>
__device__ __forceinline__ void geo_kernel_body(const typename Sto<S>::T *src,
                                                typename Sto<S>::T *dst, const StepParams &p)
{
    using R = typename Sto<S>::R;
    R mon[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    R fo[3] = {R(0), R(0), R(0)};
    size_t bid;
    if (p.nlist) {
        // one thread per listed node (rows mixed within a warp: general axes)
        bid = (size_t)p.part_base + blockIdx.x;
        const int i = blockIdx.x * blockDim.x + threadIdx.x;
        if constexpr (MON == 0) {
            if (i >= p.nlist_len)
                return;
        }
        if (i < p.nlist_len) {
            const int n = p.nlist[i];
            const int x = n % p.nx, row = n / p.nx;
            geo_node<L, S, MODEL, FORCE, MON, false>(src, dst, p, x, row % p.ny, row / p.ny, mon,
                                                     fo);
        }
    } else {
        bid = grid_block_index();
        const int x = blockIdx.x * blockDim.x + threadIdx.x;
        const int y = blockIdx.y, z = blockIdx.z;
        if constexpr (MON == 0) {
            if (x >= p.nx)
                return;
        }
        if (x < p.nx) {
            const bool interior = y > 0 && y < p.ny - 1 && (L::D == 2 || (z > 0 && z < p.nz - 1));
            if (interior)
                geo_node<L, S, MODEL, FORCE, MON, true>(src, dst, p, x, y, z, mon, fo);
            else
                geo_node<L, S, MODEL, FORCE, MON, false>(src, dst, p, x, y, z, mon, fo);
        }
    }
    if constexpr (MON == 1)
        block_monitor(mon, p.partials, bid);
    if constexpr (MON == 2) {
        R v[6] = {fo[0], fo[1], fo[2], R(0), R(0), R(0)};
        block_monitor(v, p.partials, bid);
    }
}

template <class L, int S, int MODEL, bool FORCE, int MON>
__global__ void __launch_bounds__(256) k_step_geo(const typename Sto<S>::T *src,
                                                  typename Sto<S>::T *dst, const StepParams p)
{
    geo_kernel_body<L, S, MODEL, FORCE, MON>(src, dst, p);
}

// The general kernel held to three blocks per SM (FP32 and 16-bit storage;
// unbounded the D3Q27 form takes 88-90 registers, two blocks per SM, and its
// node-list launch is memory-latency bound).  D3Q27 with 16-bit storage: four
// (64 registers; with the paired bulk kernel at seven, the 512x128x128 sphere
// step went from 0.266 to 0.263 ms).
template <class L, int S>
constexpr int kGeoMinBlocks = (L::Q == 27 && (S == ST_F16S || S == ST_BF16S)) ? 4 : 3;
template <class L, int S, int MODEL, bool FORCE, int MON>
__global__ void __launch_bounds__(256, (kGeoMinBlocks<L, S>))
    k_step_geo_bounded(const typename Sto<S>::T *src, typename Sto<S>::T *dst, const StepParams p)
{
    geo_kernel_body<L, S, MODEL, FORCE, MON>(src, dst, p);
}

// flags[n] = 1 for the nodes the plain kernel cannot update (needs_general);
// with `pairs` (nx even, the paired kernel) both nodes of such a pair.
template <class L>
__global__ void __launch_bounds__(256) k_node_flags(unsigned char *flags, const StepParams p,
                                                    bool pairs)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.nx)
        return;
    const int n = x + p.nx * (y + p.ny * z);
    const bool g = needs_general(p, n, x, y, z) || (pairs && needs_general(p, n ^ 1, x ^ 1, y, z));
    flags[n] = g ? 1 : 0;
}

// Link words from a solid mask: bit 31 = the node is solid; bit a = the
// population entering the (fluid) node along e_a would come from a solid
// node (after the face rules; wall, inlet and outflow links never do).
// count += number of solid nodes.
template <class L>
__global__ void __launch_bounds__(256) k_links(const unsigned char *solid, unsigned *links,
                                               unsigned long long *count, const StepParams p)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.nx)
        return;
    const int n = x + p.nx * (y + p.ny * z);
    unsigned w = 0u;
    if (solid[n]) {
        w = kSolidBit;
        atomicAdd(count, 1ull);
    } else {
        AxisG X, Y, Z;
        geo_axes<L>(p, x, y, z, false, X, Y, Z);
        SFor<0, L::Q>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            int off, slot;
            unsigned kind;
            link_of<L, a>(X, Y, Z, off, kind, slot);
            if (!(kind & (SK_BOUNCE | SK_OUT | SK_NODAL)) && solid[n + off])
                w |= 1u << a;
        });
    }
    links[n] = w;
}

}  // namespace lbm
