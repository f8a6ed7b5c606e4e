// lbm_pair.cuh -- the fused step for 16-bit storage with two nodes per thread.
//
// Same arithmetic as k_step (lbm_kernels.cuh).  With 2-byte values, one value
// per thread per slot makes every warp access 64 bytes, and HBM throughput
// saturates well below the copy peak; here each thread owns the nodes x and
// x+1 (x even) and moves one 32-bit word (two values) per slot.  Directions
// with e_x = +-1 are realigned in registers: a thread loads the aligned word
// holding its own positions and takes the missing half from its neighbour
// lane with a warp shuffle (lanes at the warp edge load it, positions beyond
// the row end take the wall or periodic value).  Pushed stores of the AA
// pattern are realigned the same way, and a value is written with a 16-bit
// store exactly where the aligned word would straddle two warps or the row
// end, so no thread writes a location another thread owns.
//
// Ownership (AA pattern, in place): node x reads and writes only the slot
// locations it owns, (x - e_a, abar) before and (x + e_a, a) after.  An
// aligned 32-bit load may also fetch a half owned by a node of another warp;
// that half is never used.  Inside a warp the shuffles order every lane's
// loads before any lane's stores.
//
// Both nodes of a thread are collided together in packed FP32 arithmetic
// (two lanes per instruction: __fadd2_rn, __fmul2_rn, __ffma2_rn), with
// exactly the rounding sequence of the scalar collide(), so the results are
// bitwise those of the one-node-per-thread kernel.
//
// Preconditions checked by the host: 16-bit storage, nx even.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

// ---- packed FP32 (two nodes) -------------------------------------------------
// Written as PTX with an explicit .rn rounding modifier, which forbids the
// assembler from fusing a multiply into a following add: each operation
// rounds exactly like its scalar __f*_rn counterpart in collide().
__device__ __forceinline__ unsigned long long pk(float2 v)
{
    unsigned long long r;
    memcpy(&r, &v, 8);
    return r;
}
__device__ __forceinline__ float2 upk(unsigned long long r)
{
    float2 v;
    memcpy(&v, &r, 8);
    return v;
}
__device__ __forceinline__ float2 v_add(float2 a, float2 b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 v_sub(float2 a, float2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 v_mul(float2 a, float2 b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 v_fma(float2 a, float2 b, float2 c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
    return upk(d);
}
__device__ __forceinline__ float2 v_bc(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 v_neg(float2 a) { return make_float2(-a.x, -a.y); }

template <int S>
__device__ __forceinline__ float2 dec2(unsigned w);
template <>
__device__ __forceinline__ float2 dec2<ST_F16S>(unsigned w)
{
    __half2 h;
    memcpy(&h, &w, 4);
    return __half22float2(h);
}
template <>
__device__ __forceinline__ float2 dec2<ST_BF16S>(unsigned w)
{
    __nv_bfloat162 h;
    memcpy(&h, &w, 4);
    return __bfloat1622float2(h);
}
template <int S>
__device__ __forceinline__ unsigned enc2(float2 v);
template <>
__device__ __forceinline__ unsigned enc2<ST_F16S>(float2 v)
{
    const __half2 h = __float22half2_rn(v);
    unsigned w;
    memcpy(&w, &h, 4);
    return w;
}
template <>
__device__ __forceinline__ unsigned enc2<ST_BF16S>(float2 v)
{
    const __nv_bfloat162 h = __float22bfloat162_rn(v);
    unsigned w;
    memcpy(&w, &h, 4);
    return w;
}

// collide() of lbm_kernels.cuh on two nodes at once, operation for operation,
// on the stored words: W[a] holds the two nodes' 16-bit values of direction
// a and is rewritten with the post-collision values.  The populations are
// kept packed (one register per direction instead of two) and decoded again
// where they are used: decoding is exact, so the results are those of
// collide() bit for bit, with about Q registers fewer live through the moment
// pass.  `top`: the pair lies on the row next to the moving wall, whose e_y =
// -1 populations carry the lid term (added at every decode, as the scalar
// kernel adds it once).
template <class L, int S, int MODEL, bool FORCE>
__device__ __forceinline__ void collide2w(unsigned (&W)[L::Q], bool top, const float2 (&F)[3],
                                          const Coef<float> &c, float2 (&u_out)[3],
                                          float2 &s_out, float2 &rho_out)
{
    constexpr bool COMP = MODEL == M_COMP;
    constexpr int H = L::Q / 2;
    auto g = [&](auto A_) -> float2 {
        constexpr int a = decltype(A_)::value;
        float2 v = dec2<S>(W[a]);
        if constexpr (L::e(a, 1) == -1) {
            if (top)
                v = v_add(v, v_bc(c.lid[a]));
        }
        return v;
    };
    float2 s = g(std::integral_constant<int, H>{});
    float2 j[3] = {v_bc(0.f), v_bc(0.f), v_bc(0.f)};
    SFor<0, H>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        const float2 ga = g(A_), gb = g(std::integral_constant<int, opp<L>(a)>{});
        const float2 sp = v_add(ga, gb), sm = v_sub(ga, gb);
        s = v_add(s, sp);
        SFor<0, 3>::run([&](auto K_) {
            constexpr int k = decltype(K_)::value;
            if constexpr (L::e(a, k) == 1)
                j[k] = v_add(j[k], sm);
            else if constexpr (L::e(a, k) == -1)
                j[k] = v_sub(j[k], sm);
        });
    });
    float2 rho, ir;
    if constexpr (COMP) {
        rho = v_add(s, v_bc(c.sigma));
        ir = make_float2(1.f / rho.x, 1.f / rho.y);
    } else {
        rho = v_bc(c.rho0);
        ir = v_bc(c.inv_rho0);
    }
    s_out = s;
    rho_out = rho;
    float2 u[3], jf[3];
    SFor<0, 3>::run([&](auto K_) {
        constexpr int k = decltype(K_)::value;
        if constexpr (FORCE)
            jf[k] = v_fma(v_bc(0.5f), F[k], j[k]);
        else
            jf[k] = j[k];
        u[k] = v_mul(jf[k], ir);
    });
    const float2 uu = v_fma(u[2], u[2], v_fma(u[1], u[1], v_mul(u[0], u[0])));
    float2 A = v_fma(v_mul(v_bc(-1.5f), rho), uu, s);
    if constexpr (FORCE) {
        const float2 uF = v_fma(u[2], F[2], v_fma(u[1], F[1], v_mul(u[0], F[0])));
        A = v_fma(v_bc(__fmul_rn(-3.f, c.kf)), uF, A);
    }
    const float2 r3 = v_mul(v_bc(3.f), rho), r45 = v_mul(v_bc(4.5f), rho);
    const float2 om = v_bc(c.omega);
    // same operations, in the same order, as the scalar collide()
    auto pair_eq = [&](auto A_, float2 &sym, float2 &asym) {
        constexpr int a = decltype(A_)::value;
        float2 ej = v_bc(0.f), eF = v_bc(0.f);
        (void)eF;
        SFor<0, 3>::run([&](auto K_) {
            constexpr int k = decltype(K_)::value;
            if constexpr (L::e(a, k) == 1) {
                ej = v_add(ej, jf[k]);
                if constexpr (FORCE)
                    eF = v_add(eF, F[k]);
            } else if constexpr (L::e(a, k) == -1) {
                ej = v_sub(ej, jf[k]);
                if constexpr (FORCE)
                    eF = v_sub(eF, F[k]);
            }
        });
        const float2 eu = v_mul(ej, ir);
        sym = v_fma(v_mul(r45, eu), eu, A);
        asym = v_mul(r3, eu);
        if constexpr (FORCE) {
            sym = v_fma(v_mul(v_bc(__fmul_rn(9.f, c.kf)), eu), eF, sym);
            asym = v_fma(v_bc(__fmul_rn(3.f, MODEL == M_TRT ? c.kf_m : c.kf)), eF, asym);
        }
    };
    if constexpr (MODEL == M_TRT) {
        const float2 omm = v_bc(c.omega_m);
        SFor<0, H>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            constexpr int b = opp<L>(a);
            const float2 t = v_bc(float(L::w(a)));
            float2 sym, asym;
            pair_eq(A_, sym, asym);
            const float2 ga = g(A_), gb = g(std::integral_constant<int, b>{});
            const float2 hp = v_mul(v_add(ga, gb), v_bc(0.5f));
            const float2 hm = v_mul(v_sub(ga, gb), v_bc(0.5f));
            const float2 gp = v_fma(om, v_fma(sym, t, v_neg(hp)), hp);
            const float2 gm =
                v_fma(omm, v_fma(asym, v_bc(w_lo<L>(a)), v_fma(asym, t, v_neg(hm))), hm);
            W[a] = enc2<S>(v_add(gp, gm));
            W[b] = enc2<S>(v_sub(gp, gm));
        });
    } else {
        SFor<0, H>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            constexpr int b = opp<L>(a);
            const float2 t = v_bc(float(L::w(a)));
            float2 sym, asym;
            pair_eq(A_, sym, asym);
            const float2 at = v_fma(asym, t, v_mul(asym, v_bc(w_lo<L>(a))));
            const float2 fa = v_fma(sym, t, at), fb = v_fma(sym, t, v_neg(at));
            const float2 ga = g(A_), gb = g(std::integral_constant<int, b>{});
            W[a] = enc2<S>(v_fma(om, v_sub(fa, ga), ga));
            W[b] = enc2<S>(v_fma(om, v_sub(fb, gb), gb));
        });
    }
    {
        const float2 t0 = v_bc(float(L::w(H)));
        const float2 gH = g(std::integral_constant<int, H>{});
        W[H] = enc2<S>(v_fma(om, v_fma(t0, A, v_neg(gH)), gH));
    }
    u_out[0] = u[0];
    u_out[1] = u[1];
    u_out[2] = u[2];
}

constexpr int kPairThreads = 128;  // threads per block; 256 nodes per block

__device__ __forceinline__ unsigned lo16(unsigned w) { return w & 0xffffu; }
__device__ __forceinline__ unsigned hi16(unsigned w) { return w >> 16; }
// (hi half of a, lo half of b) as (lo, hi) of the result
__device__ __forceinline__ unsigned join_hi_lo(unsigned a, unsigned b)
{
    return __byte_perm(a, b, 0x5432);
}

// Source (pull) or target (push) row of direction a for row (y, z): the row
// shifted by -e_a (pull) or +e_a (push) in y and z, wrapped on periodic axes;
// `wall` when that row lies beyond a y or z wall.
template <class L, int a, int SIGN, bool IROW = false>
__device__ __forceinline__ int shifted_row(const StepParams &p, int y, int z, bool &wall)
{
    constexpr int ey = SIGN * L::e(a, 1), ez = SIGN * L::e(a, 2);
    int ys = y + ey, zs = z + ez;
    wall = false;
    if constexpr (IROW)  // y and z have neighbours on both sides
        return ys + p.ny * zs;
    if (ys < 0 || ys >= p.ny) {
        if (p.periodic & 2)
            ys = ys < 0 ? ys + p.ny : ys - p.ny;
        else
            wall = true;
    }
    if (zs < 0 || zs >= p.nz) {
        if (p.periodic & 4)
            zs = zs < 0 ? zs + p.nz : zs - p.nz;
        else
            wall = true;
    }
    return ys + p.ny * zs;
}

// SKIP (pull scheme only): a box with per-face boundaries or obstacles; pairs
// with a node that needs the general kernel are loaded (their words feed the
// neighbour lanes' realignment) but neither collided nor stored.
template <class L, int S, int PAT, int MODEL, bool FORCE, bool IROW, bool RED, bool SKIP = false>
__device__ __forceinline__ void pair_body(const unsigned short *src, unsigned short *dst,
                                          const StepParams &p)
{
    using R = float;
    constexpr int Q = L::Q;
    const Coef<R> &c = p.cf;
    const size_t N = (size_t)p.N;
    const int nx = p.nx;
    const int lane = threadIdx.x & 31;
    const int x = 2 * (blockIdx.x * kPairThreads + threadIdx.x);
    const int y = blockIdx.y, z = blockIdx.z;
    const bool active = x < nx;
    const int row = y + p.ny * z;
    const size_t n = (size_t)row * nx + x;  // even
    const bool xper = p.periodic & 1;
    const bool top = p.lid_on && (y == p.ny - 1);
    bool own = active;  // this pair is collided and stored here
    // interior rows: the warp-edge cases as per-thread predicates, fixed for
    // the whole step; the row ends (x = 0, x + 2 = nx: at most two warps of a
    // row) are fixed up behind one warp-uniform flag in the AA push stores
    // Two forms of the interior rows' loads, bitwise identical: the row ends
    // as per-lane conditions inside each direction, or fixed up behind a
    // warp-uniform flag (measured faster for the D3Q19 AA gather only).
    constexpr bool kUniformRowEnd = L::Q == 19 && PAT == PAT_GATHER;
    const bool first = x == 0, last_pair = x + 2 == nx;
    const bool row_end = __any_sync(0xffffffffu, first || last_pair);
    const bool ld_xp = active && lane == 0 && !first;       // e_x = +1: word before the warp
    const bool ld_xm = active && lane == 31 && !last_pair;  // e_x = -1: word after the warp
    (void)row_end;
    (void)ld_xp;
    (void)ld_xm;
    if constexpr (SKIP) {
        static_assert(PAT == PAT_PULL, "the pull scheme only");
        if (active)
            own = !needs_general(p, (int)n, x, y, z) && !needs_general(p, (int)n + 1, x + 1, y, z);
    }

    auto word = [&](const unsigned short *base, size_t i) -> unsigned {
        return *reinterpret_cast<const unsigned *>(base + i);
    };
    const unsigned short *src_n = src + n;
    unsigned short *dst_n = dst + n;

    // ---- gather the incoming pairs -------------------------------------------
    // Phase 1 issues every load (aligned words, the warp-edge words, the
    // wall/periodic values at the row ends) before any shuffle, so that all
    // of them are in flight together; phase 2 realigns with shuffles.
    unsigned W[Q], Wx[Q];  // Wx: the extra word (warp edge) or row-end value
    SFor<0, Q>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        constexpr int b = opp<L>(a);
        constexpr int ex = L::e(a, 0);
        Wx[a] = 0u;
        if constexpr (PAT == PAT_LOCAL) {
            W[a] = active ? word(src, (size_t)a * N + n) : 0u;
            return;
        }
        // pull side: slot `ns` of the row shifted by -e_a, or the bounce
        // slot `bs` of the node itself beyond a wall
        constexpr int ns = (PAT == PAT_PULL) ? a : b;
        constexpr int bs = (PAT == PAT_PULL) ? b : a;
        if constexpr (IROW && kUniformRowEnd) {
            // q: position x of slot ns in the row shifted by -e_a; lane 0 (31)
            // also loads the word before (after) the warp's span for e_x = +1 (-1)
            const unsigned short *q = src_n + (PAT == PAT_PULL ? p.pull_off[a] : p.push_off[b]);
            if (active)
                W[a] = word(q, 0);
            if constexpr (ex == 1) {
                if (ld_xp)
                    Wx[a] = *reinterpret_cast<const unsigned *>(q - 2);
            } else if constexpr (ex == -1) {
                if (ld_xm)
                    Wx[a] = word(q, 2);
            }
            return;
        }
        if constexpr (IROW) {
            // q: position x of slot ns in the row shifted by -e_a
            const unsigned short *q = src_n + (PAT == PAT_PULL ? p.pull_off[a] : p.push_off[b]);
            W[a] = active ? word(q, 0) : 0u;
            if constexpr (ex == 1) {
                if (active && x == 0)
                    Wx[a] = xper ? q[nx - 1] : src_n[(size_t)bs * N];
                else if (active && lane == 0)
                    Wx[a] = *reinterpret_cast<const unsigned *>(q - 2);
            } else if constexpr (ex == -1) {
                if (active && x + 2 == nx)
                    Wx[a] = xper ? q[-x] : src_n[(size_t)bs * N + 1];
                else if (active && lane == 31)
                    Wx[a] = word(q, 2);
            }
            return;
        }
        bool yzw;
        const int srow = shifted_row<L, a, -1, IROW>(p, y, z, yzw);
        if (ex == 0 || yzw) {
            W[a] = active ? word(src, (size_t)(yzw ? bs : ns) * N + (yzw ? n : (size_t)srow * nx + x))
                          : 0u;
            return;
        }
        const unsigned short *rbase = src + (size_t)ns * N + (size_t)srow * nx;
        W[a] = active ? word(rbase, x) : 0u;
        if constexpr (ex == 1) {
            if (active && x == 0)  // position -1: periodic wrap or bounce-back
                Wx[a] = xper ? rbase[nx - 1] : src[(size_t)bs * N + n];
            else if (active && lane == 0)  // positions (x-2, x-1) lie in the previous warp's span
                Wx[a] = word(rbase, x - 2);
        } else {
            if (active && x + 2 == nx)  // position nx: periodic wrap or bounce-back
                Wx[a] = xper ? rbase[0] : src[(size_t)bs * N + n + 1];
            else if (active && lane == 31)  // positions (x+2, x+3) lie in the next warp's span
                Wx[a] = word(rbase, x + 2);
        }
    });
    if constexpr (PAT != PAT_LOCAL && IROW && kUniformRowEnd) {
        SFor<0, Q>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            constexpr int b = opp<L>(a);
            constexpr int ex = L::e(a, 0);
            constexpr int bs = (PAT == PAT_PULL) ? b : a;
            if constexpr (ex == 1) {
                // positions (x-1, x): hi of the previous word, lo of W
                const unsigned wp = __shfl_up_sync(0xffffffffu, W[a], 1);
                W[a] = join_hi_lo(lane == 0 ? Wx[a] : wp, W[a]);
                if (row_end && first) {  // position -1: periodic image or wall (own slot bs)
                    const unsigned short *q =
                        src_n + (PAT == PAT_PULL ? p.pull_off[a] : p.push_off[b]);
                    const unsigned e = xper ? q[nx - 1] : src_n[(size_t)bs * N];
                    W[a] = (W[a] & 0xffff0000u) | e;
                }
            } else if constexpr (ex == -1) {
                // positions (x+1, x+2): hi of W, lo of the next word
                const unsigned wn = __shfl_down_sync(0xffffffffu, W[a], 1);
                W[a] = join_hi_lo(W[a], lane == 31 ? Wx[a] : wn);
                if (row_end && last_pair) {  // position nx: periodic image or wall
                    const unsigned short *q =
                        src_n + (PAT == PAT_PULL ? p.pull_off[a] : p.push_off[b]);
                    const unsigned e = xper ? q[-x] : src_n[(size_t)bs * N + 1];
                    W[a] = (W[a] & 0x0000ffffu) | (e << 16);
                }
            }
        });
    } else if constexpr (PAT != PAT_LOCAL) {
        SFor<0, Q>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            constexpr int ex = L::e(a, 0);
            if constexpr (ex != 0) {
                bool yzw;
                (void)shifted_row<L, a, -1, IROW>(p, y, z, yzw);
                if (yzw)
                    return;  // block-uniform
                const unsigned w0 = W[a];
                if constexpr (ex == 1) {
                    // positions (x-1, x): hi of the previous word, lo of w0
                    unsigned wp = __shfl_up_sync(0xffffffffu, w0, 1);
                    if (lane == 0)
                        wp = Wx[a];
                    unsigned pr = join_hi_lo(wp, w0);
                    if (x == 0)
                        pr = (pr & 0xffff0000u) | Wx[a];
                    W[a] = pr;
                } else {
                    // positions (x+1, x+2): hi of w0, lo of the next word
                    unsigned wn = __shfl_down_sync(0xffffffffu, w0, 1);
                    if (lane == 31)
                        wn = Wx[a];
                    unsigned pr = join_hi_lo(w0, wn);
                    if (x + 2 == nx)
                        pr = (pr & 0x0000ffffu) | (Wx[a] << 16);
                    W[a] = pr;
                }
            }
        });
    }

    float mon[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    // ---- collide nodes x and x+1 together (packed FP32) ------------------------
    if (own) {
        float2 F[3] = {v_bc(0.f), v_bc(0.f), v_bc(0.f)};
        if constexpr (FORCE) {
            for (int k = 0; k < L::D; ++k)
                F[k] = *reinterpret_cast<const float2 *>(p.F + k * N + n);
        }
        float2 u2[3], s2, rho2;
        collide2w<L, S, MODEL, FORCE>(W, top, F, c, u2, s2, rho2);
        if constexpr (RED) {  // the two nodes' monitor values, summed in the thread
            float m0[6], m1[6];
            const float ua[3] = {u2[0].x, u2[1].x, u2[2].x}, ub[3] = {u2[0].y, u2[1].y, u2[2].y};
            monitor_values(s2.x, rho2.x, ua, m0);
            monitor_values(s2.y, rho2.y, ub, m1);
            for (int k = 0; k < 5; ++k)
                mon[k] = o_add(m0[k], m1[k]);
            mon[5] = fmaxf(m0[5], m1[5]);
        }
    }

    // ---- store ---------------------------------------------------------------
    auto put_word = [&](size_t i, unsigned w) { *reinterpret_cast<unsigned *>(dst + i) = w; };
    SFor<0, Q>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        constexpr int b = opp<L>(a);
        constexpr int ex = L::e(a, 0);
        const unsigned O = W[a];
        if constexpr (PAT == PAT_PULL) {
            if (own)
                put_word((size_t)a * N + n, O);
            return;
        }
        if constexpr (PAT == PAT_LOCAL) {
            if (active)
                put_word((size_t)b * N + n, O);
            return;
        }
        // AA push of f*_a to x + e_a (slot a); beyond a wall: slot b of the node
        if constexpr (IROW) {
            // q: position x of slot a in the row shifted by +e_a
            unsigned short *q = dst_n + p.push_st[a];
            if constexpr (ex == 0) {
                if (active)
                    *reinterpret_cast<unsigned *>(q) = O;
            } else if constexpr (ex == 1) {
                // targets (x+1, x+2): the aligned word (x+2, x+3) takes this
                // lane's hi and the next lane's lo; lane 0 writes x+1 alone, lane
                // 31 x+2 alone; the row's last pair pushes x+2 = nx beyond the end
                const unsigned On = __shfl_down_sync(0xffffffffu, O, 1);
                if (active && lane != 31 && !last_pair)
                    *reinterpret_cast<unsigned *>(q + 2) = join_hi_lo(O, On);
                if (active && lane == 0)
                    q[1] = (unsigned short)lo16(O);
                if (ld_xm)
                    q[2] = (unsigned short)hi16(O);
                if (row_end && active && last_pair) {
                    if (xper)
                        q[-x] = (unsigned short)hi16(O);
                    else
                        dst_n[(size_t)b * N + 1] = (unsigned short)hi16(O);
                }
            } else {
                // targets (x-1, x): the aligned word (x-2, x-1) takes the
                // previous lane's hi and this lane's lo; lane 0 writes x-1 alone
                // (x = 0: beyond the row start), the warp's or row's last pair x
                const unsigned Op = __shfl_up_sync(0xffffffffu, O, 1);
                if (active && lane != 0)
                    *reinterpret_cast<unsigned *>(q - 2) = join_hi_lo(Op, O);
                if (ld_xp)
                    q[-1] = (unsigned short)lo16(O);
                if (active && (lane == 31 || last_pair))
                    q[0] = (unsigned short)hi16(O);
                if (row_end && active && first) {
                    if (xper)
                        q[nx - 1] = (unsigned short)lo16(O);
                    else
                        dst_n[(size_t)b * N] = (unsigned short)lo16(O);
                }
            }
            return;
        }
        bool yzw;
        const int trow = shifted_row<L, a, +1, IROW>(p, y, z, yzw);
        if (ex == 0 || yzw) {
            if (active)
                put_word(yzw ? (size_t)b * N + n : (size_t)a * N + (size_t)trow * nx + x, O);
            return;
        }
        unsigned short *rbase = dst + (size_t)a * N + (size_t)trow * nx;
        if constexpr (ex == 1) {
            // targets (x+1, x+2); this lane writes the aligned word (x+2, x+3)
            const unsigned On = __shfl_down_sync(0xffffffffu, O, 1);
            if (!active)
                return;
            const bool last = lane == 31 || x + 2 >= nx;  // neighbour lane not in this row span
            if (lane == 0)
                rbase[x + 1] = (unsigned short)lo16(O);
            if (x + 2 < nx) {
                if (last)
                    rbase[x + 2] = (unsigned short)hi16(O);
                else
                    put_word((size_t)a * N + (size_t)trow * nx + x + 2, join_hi_lo(O, On));
            } else {  // node x+1 = nx-1 pushes beyond the row end
                if (xper)
                    rbase[0] = (unsigned short)hi16(O);
                else
                    dst[(size_t)b * N + n + 1] = (unsigned short)hi16(O);
            }
        } else {
            // targets (x-1, x); this lane writes the aligned word (x-2, x-1)
            const unsigned Op = __shfl_up_sync(0xffffffffu, O, 1);
            if (!active)
                return;
            const bool last = lane == 31 || x + 2 >= nx;
            if (x == 0) {  // node 0 pushes beyond the row start
                if (xper)
                    rbase[nx - 1] = (unsigned short)lo16(O);
                else
                    dst[(size_t)b * N + n] = (unsigned short)lo16(O);
            } else if (lane == 0) {
                rbase[x - 1] = (unsigned short)lo16(O);
            } else {
                put_word((size_t)a * N + (size_t)trow * nx + x - 2, join_hi_lo(Op, O));
            }
            if (last)
                rbase[x] = (unsigned short)hi16(O);
        }
    });
    if constexpr (RED)
        block_monitor(mon, p.partials, grid_block_index());
}

// ---- moments + FP64 reduction, 16-bit storage, two nodes per thread ------------
// k_moments for the LOCAL and SWAPPED forms (each node's own slots) with one
// 32-bit load per slot for two adjacent nodes.  Per node the values are those
// of k_moments (moments_of, monitor_values), and so is every FP32 sum over a
// group of 32 consecutive nodes of a row segment: the one-node kernel's warp
// butterfly (xor 16, 8, 4, 2, 1 over the node index) is node 2t+h of the
// group = half h of lane t, i.e. xor 8, 4, 2, 1 over the lanes of each half
// warp and, last, the thread's two halves.  Only the FP64 accumulation of the
// group sums runs in another order.  Grid-stride over segments of 256 nodes;
// block b writes partials[b].  nx even.
template <class L, int S, int FORM, bool COMP, bool FORCE>
__global__ void __launch_bounds__(kPairThreads) k_moments_pair(const unsigned short *src,
                                                              const StepParams p,
                                                              const MomParams m)
{
    static_assert(FORM == FORM_LOCAL || FORM == FORM_SWAPPED, "the node's own slots only");
    using R = float;
    constexpr int Q = L::Q;
    const Coef<R> &c = p.cf;
    const size_t N = (size_t)p.N;
    const int lane = threadIdx.x & 31;
    // lane k < 5 of each half warp keeps the FP64 running sum of monitor value
    // k of its 32-node group (one FP64 add per warp and segment); the maximum
    // stays in FP32, where it is exact
    double acc = 0.0;
    R accmax = R(0);
    const int hk = lane & 15;
    for (int seg = blockIdx.x; seg < m.nseg; seg += gridDim.x) {
        const int xs = seg % m.xseg;
        const int row = seg / m.xseg;
        const int y = row % p.ny, z = row / p.ny;
        const int x = xs * (2 * kPairThreads) + 2 * threadIdx.x;
        const bool active = x < p.nx;
        const int n0 = x + p.nx * (y + p.ny * z);
        unsigned W[Q];
        SFor<0, Q>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            constexpr int slot = FORM == FORM_LOCAL ? a : opp<L>(a);
            W[a] = active ? *reinterpret_cast<const unsigned *>(src + (size_t)slot * N + n0) : 0u;
        });
        R vals[2][kReduceVals];
        for (int h = 0; h < 2; ++h) {
            for (int k = 0; k < kReduceVals; ++k)
                vals[h][k] = R(0);
            const int n = n0 + h;
            const bool solid = active && m.links && (m.links[n] >> 31);
            if (solid) {
                if (m.p_out) {
                    if (m.out_f32)
                        ((float *)m.p_out)[n] = 0.f;
                    else
                        ((double *)m.p_out)[n] = 0.0;
                }
                if (m.u_out) {
                    for (int k = 0; k < L::D; ++k) {
                        if (m.out_f32)
                            ((float *)m.u_out)[k * N + n] = 0.f;
                        else
                            ((double *)m.u_out)[k * N + n] = 0.0;
                    }
                }
            }
            if (active && !solid) {
                R g[Q];
                SFor<0, Q>::run([&](auto A_) {
                    constexpr int a = decltype(A_)::value;
                    const float2 v = dec2<S>(W[a]);
                    g[a] = h ? v.y : v.x;
                });
                R s_, rho, u[3];
                moments_of<L, R, COMP, FORCE>(g, p, n, s_, rho, u);
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
                monitor_values(s_, rho, u, vals[h]);
            }
        }
        if (m.partials) {
            R mine = R(0);
#pragma unroll
            for (int k = 0; k < kReduceVals; ++k) {
                R v0 = vals[0][k], v1 = vals[1][k];
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) {
                    const R w0 = __shfl_xor_sync(0xffffffffu, v0, o);
                    const R w1 = __shfl_xor_sync(0xffffffffu, v1, o);
                    if (k == 5) {
                        v0 = max(v0, w0);
                        v1 = max(v1, w1);
                    } else {
                        v0 += w0;
                        v1 += w1;
                    }
                }
                // the 32-node group's value
                if (k == 5)
                    accmax = max(accmax, max(v0, v1));
                else
                    mine = hk == k ? v0 + v1 : mine;
            }
            if (hk < 5)
                acc += double(mine);
        }
    }
    if (!m.partials)
        return;
    __shared__ double sh[2 * kPairThreads / 32][kReduceVals];
    const int grp = threadIdx.x >> 4;  // 32-node group of the block
    if (hk < 5)
        sh[grp][hk] = acc;
    else if (hk == 5)
        sh[grp][5] = double(accmax);
    __syncthreads();
    if (threadIdx.x < kReduceVals) {
        const int k = threadIdx.x;
        double r = sh[0][k];
        for (int i = 1; i < 2 * kPairThreads / 32; ++i)
            r = (k == 5) ? fmax(r, sh[i][k]) : r + sh[i][k];
        m.partials[blockIdx.x * kPartialStride + k] = r;
    }
}

// The pull step of a box with per-face boundaries or obstacles on the pairs
// the paired kernel can update (see k_step_skip).  MON: 0, 1 = monitor sums,
// 2 = obstacle force (zero here).  Blocks per SM: D3Q27 seven (72 registers,
// as the paired D3Q27 pull; eight spilled 356 bytes and was 16 % slower on the
// sphere), D3Q19 six.
template <class L>
constexpr int kPairSkipMinBlocks = L::Q == 27 ? 7 : 6;
template <class L, int S, int MODEL, bool FORCE, int MON>
__global__ void __launch_bounds__(kPairThreads, (kPairSkipMinBlocks<L>))
    k_step_pair_skip(const unsigned short *src, unsigned short *dst, const StepParams p)
{
    if constexpr (MON == 2) {
        if (threadIdx.x < kReduceVals)
            p.partials[grid_block_index() * kPartialStride + threadIdx.x] = 0.0;
    }
    const int y = blockIdx.y, z = blockIdx.z;
    const bool irow = y > 0 && y < p.ny - 1 && (L::D == 2 || (z > 0 && z < p.nz - 1));
    if (irow)
        pair_body<L, S, PAT_PULL, MODEL, FORCE, true, MON == 1, true>(src, dst, p);
    else
        pair_body<L, S, PAT_PULL, MODEL, FORCE, false, MON == 1, true>(src, dst, p);
}

// The paired step held to MINB blocks per SM (the launcher's measured
// choice per lattice and pattern): without the bound the compiler takes more
// registers than these memory-latency-bound kernels can afford.
template <class L, int S, int PAT, int MODEL, bool FORCE, int MINB>
__global__ void __launch_bounds__(kPairThreads, MINB) k_step_pair_bounded(const unsigned short *src,
                                                                          unsigned short *dst,
                                                                          const StepParams p)
{
    const int y = blockIdx.y, z = blockIdx.z;
    const bool irow = y > 0 && y < p.ny - 1 && (L::D == 2 || (z > 0 && z < p.nz - 1));
    if (irow || PAT == PAT_LOCAL)
        pair_body<L, S, PAT, MODEL, FORCE, true, false>(src, dst, p);
    else
        pair_body<L, S, PAT, MODEL, FORCE, false, false>(src, dst, p);
}

template <class L, int S, int PAT, int MODEL, bool FORCE, bool RED = false>
__global__ void __launch_bounds__(kPairThreads) k_step_pair(const unsigned short *src,
                                                            unsigned short *dst, const StepParams p)
{
    const int y = blockIdx.y, z = blockIdx.z;
    const bool irow = y > 0 && y < p.ny - 1 && (L::D == 2 || (z > 0 && z < p.nz - 1));
    if (irow || PAT == PAT_LOCAL)
        pair_body<L, S, PAT, MODEL, FORCE, true, RED>(src, dst, p);
    else
        pair_body<L, S, PAT, MODEL, FORCE, false, RED>(src, dst, p);
}

}  // namespace lbm
