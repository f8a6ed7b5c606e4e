// lbm_adjoint.cuh -- reverse (adjoint) collide-stream kernels.
//
// Not in the paper: the exact transpose of one IMEXLBM step, used for
// gradients of J = rho0/2 sum_x |u(x, T)|^2 with respect to the body-force
// field F and the moving-wall velocity U (incompressible model).
//
// With f^{k+1} = S(C(f^k)) (C: collision of Eq. (collision) with the Guo
// source; S: bounce-back + propagation, affine in U) and lambda^k = dJ/df^k:
//   mu^k      = S^T lambda^{k+1}:  mu_b(x) = lambda_b(x + e_b), or
//               lambda_bbar(x) when x + e_b lies beyond a wall;
//   lambda^k  = (dC/df)^T mu^k at node x, which only needs u^k(x):
//               lambda_b = (1-omega) mu_b + omega s + e_b . a,
//               a = omega (3v + 9w - 3 u s) + (1 - omega/2)(9z - 3 F s)/rho0,
//   dJ/dF(x) += (3v + 9w - 3 u s) + (1 - omega/2)(9z - 3 F s)/(2 rho0),
//   dJ/dU    += lambda_a(x) 2 t_a rho0 e_a / c_s^2 over links crossing the lid,
// where s = sum t_a mu_a, v = sum t_a mu_a e_a, w = sum t_a mu_a (e_a.u) e_a,
// z = sum t_a mu_a (e_a.F) e_a.  The gather of mu is the pull of the forward
// kernel run backwards: every output is written by exactly one thread.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {


// INTERIOR: the node's row has neighbours inside the box in y and z (no wall,
// no wrap), so only the x axis needs per-thread boundary logic.
template <class L, class R, bool FORCE, bool INTERIOR>
__device__ __forceinline__ void adjoint_node(const StepParams &p, const AdjParams &ap, int x,
                                             int y, int z, R (&gu)[3])
{
    constexpr int Q = L::Q;
    const Coef<R> &c = coef<R>(p);
    const size_t N = (size_t)p.N;
    const int n = x + p.nx * (y + p.ny * z);
    const R *lam = (const R *)ap.lam_in;
    AxisNbr X, Y, Z;
    make_axes<L, INTERIOR>(p, x, y, z, X, Y, Z);
    const bool lid_row = !INTERIOR && p.lid_on && (y == p.ny - 1);
    R mu[Q];
    SFor<0, Q>::run([&](auto B_) {
        constexpr int b = decltype(B_)::value;
        constexpr int bb = opp<L>(b);
        int off;
        bool wall;
        upstream<L, bb>(X, Y, Z, off, wall);  // upstream of bb at x is x + e_b
        if (wall) {
            const R v = lam[bb * N + n];
            mu[b] = v;
            if constexpr (L::e(bb, 1) == -1) {
                if (lid_row) {
                    const R cw = R(6.0 * L::w(bb)) * c.rho0 * v;
                    SFor<0, 3>::run([&](auto K_) {
                        constexpr int k = decltype(K_)::value;
                        if constexpr (L::e(bb, k) != 0)
                            gu[k] += R(L::e(bb, k)) * cw;
                    });
                }
            }
        } else {
            mu[b] = lam[b * N + (n + off)];
        }
    });
    R u[3] = {R(0), R(0), R(0)}, F[3] = {R(0), R(0), R(0)};
    const R *uk = (const R *)ap.u_k;
    SFor<0, L::D>::run([&](auto K_) {
        constexpr int k = decltype(K_)::value;
        u[k] = uk[k * N + n];
        if constexpr (FORCE)
            F[k] = R(p.F[k * N + n]);
    });
    R s = R(0), v[3] = {R(0), R(0), R(0)}, w[3] = {R(0), R(0), R(0)}, zz[3] = {R(0), R(0), R(0)};
    SFor<0, Q>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        // FP32: the weight as hi + lo (see w_lo), or the momentum mode of the
        // adjoint grows by 1 + 7.45e-9 omega per reverse step
        R tm;
        if constexpr (std::is_same<R, float>::value)
            tm = wmul<L, a>(mu[a]);
        else
            tm = R(L::w(a)) * mu[a];
        s += tm;
        R eu = R(0), eF = R(0);
        (void)eF;
        SFor<0, 3>::run([&](auto K_) {
            constexpr int k = decltype(K_)::value;
            if constexpr (L::e(a, k) == 1) {
                eu += u[k];
                if constexpr (FORCE)
                    eF += F[k];
            } else if constexpr (L::e(a, k) == -1) {
                eu -= u[k];
                if constexpr (FORCE)
                    eF -= F[k];
            }
        });
        const R tmu = tm * eu;
        R tmf = R(0);
        (void)tmf;
        if constexpr (FORCE)
            tmf = tm * eF;
        SFor<0, 3>::run([&](auto K_) {
            constexpr int k = decltype(K_)::value;
            if constexpr (L::e(a, k) == 1) {
                v[k] += tm;
                w[k] += tmu;
                if constexpr (FORCE)
                    zz[k] += tmf;
            } else if constexpr (L::e(a, k) == -1) {
                v[k] -= tm;
                w[k] -= tmu;
                if constexpr (FORCE)
                    zz[k] -= tmf;
            }
        });
    });
    const R om = c.omega;
    const R half = R(1) - R(0.5) * om;
    R bvec[3], avec[3];
    SFor<0, 3>::run([&](auto K_) {
        constexpr int k = decltype(K_)::value;
        const R bk = R(3) * v[k] + R(9) * w[k] - R(3) * u[k] * s;
        R ck = R(0);
        if constexpr (FORCE)
            ck = (R(9) * zz[k] - R(3) * F[k] * s) * c.inv_rho0;
        bvec[k] = bk + R(0.5) * half * ck;
        avec[k] = om * bk + half * ck;
    });
    R *lo = (R *)ap.lam_out;
    const R base = om * s;
    const R keep = R(1) - om;
    SFor<0, Q>::run([&](auto B_) {
        constexpr int b = decltype(B_)::value;
        R ea = R(0);
        SFor<0, 3>::run([&](auto K_) {
            constexpr int k = decltype(K_)::value;
            if constexpr (L::e(b, k) == 1)
                ea += avec[k];
            else if constexpr (L::e(b, k) == -1)
                ea -= avec[k];
        });
        lo[b * N + n] = keep * mu[b] + base + ea;
    });
    R *g = (R *)ap.gF;
    SFor<0, L::D>::run([&](auto K_) {
        constexpr int k = decltype(K_)::value;
        g[k * N + n] += bvec[k];
    });
}

// grid as k_step.  Blocks on the top row (y = ny-1) also add their lid
// contribution to gU_part[(z * xseg + blockIdx.x) * 4 + k].
template <class L, class R, bool FORCE>
__device__ __forceinline__ void adjoint_kernel_body(const StepParams &p, const AdjParams &ap)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    R gu[3] = {R(0), R(0), R(0)};
    if (x < p.nx) {
        const bool interior = y > 0 && y < p.ny - 1 && (L::D == 2 || (z > 0 && z < p.nz - 1));
        if (interior)
            adjoint_node<L, R, FORCE, true>(p, ap, x, y, z, gu);
        else
            adjoint_node<L, R, FORCE, false>(p, ap, x, y, z, gu);
    }
    if (!(p.lid_on && y == p.ny - 1))
        return;  // block-uniform
    __shared__ double sh[8][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 3; ++k) {
        const R s = warp_sum(gu[k]);
        if (lane == 0)
            sh[warp][k] = double(s);
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double r = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            r += sh[w][threadIdx.x];
        ap.gU_part[((size_t)z * ap.xseg + blockIdx.x) * 4 + threadIdx.x] += r;
    }
}

template <class L, class R, bool FORCE>
__global__ void __launch_bounds__(256) k_adjoint(const StepParams p, const AdjParams ap)
{
    adjoint_kernel_body<L, R, FORCE>(p, ap);
}

// The FP32 adjoint step with a force held to MINB blocks per SM: unbounded it
// takes 63-64 registers (four blocks per SM) and is memory-latency bound.
template <class L, class R, bool FORCE, int MINB>
__global__ void __launch_bounds__(256, MINB) k_adjoint_bounded(const StepParams p,
                                                               const AdjParams ap)
{
    adjoint_kernel_body<L, R, FORCE>(p, ap);
}

// Seed at T: lambda_a = e_a . u^T, gF = u^T / 2 (the direct dJ/dF term).
template <class L, int S, bool FORCE>
__global__ void __launch_bounds__(256) k_adjoint_seed(const StepParams p, const AdjParams ap)
{
    using T = typename Sto<S>::T;
    using R = typename Sto<S>::R;
    constexpr int Q = L::Q;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.nx)
        return;
    const Coef<R> &c = coef<R>(p);
    const size_t N = (size_t)p.N;
    const int n = x + p.nx * (y + p.ny * z);
    const T *st = (const T *)ap.state;
    R j[3] = {R(0), R(0), R(0)};
    SFor<0, Q>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        const R g = Sto<S>::dec(st[a * N + n]);
        SFor<0, 3>::run([&](auto K_) {
            constexpr int k = decltype(K_)::value;
            if constexpr (L::e(a, k) == 1)
                j[k] += g;
            else if constexpr (L::e(a, k) == -1)
                j[k] -= g;
        });
    });
    R u[3];
    SFor<0, 3>::run([&](auto K_) {
        constexpr int k = decltype(K_)::value;
        R jk = j[k];
        if constexpr (FORCE) {
            if (k < L::D)
                jk -= R(0.5) * R(p.F[k * N + n]);
        }
        u[k] = jk * c.inv_rho0;
    });
    R *lam = (R *)ap.lam_out;
    SFor<0, Q>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        lam[a * N + n] = R(L::e(a, 0)) * u[0] + R(L::e(a, 1)) * u[1] + R(L::e(a, 2)) * u[2];
    });
    R *g = (R *)ap.gF;
    for (int k = 0; k < L::D; ++k)
        g[k * N + n] = R(0.5) * u[k];
}

// dJdF += gF; gF = 0 (end of a checkpoint segment).  1D grid over d*N.
template <class R>
__global__ void __launch_bounds__(256) k_adjoint_flush(R *gF, double *dJdF, size_t count)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x) {
        if (dJdF)
            dJdF[i] += double(gF[i]);
        gF[i] = R(0);
    }
}

}  // namespace lbm
