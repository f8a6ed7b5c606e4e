// lbm_lattice.cuh -- compile-time velocity sets and storage codecs.
//
// Velocity sets of Sec. 2.1 (arxiv 2201.11330).  D2Q9 follows the table the
// paper prints: direction a = 3*(e_x+1) + (e_y+1), e_x slowest.  D3Q19 and
// D3Q27 use the same lexicographic rule over (e_x, e_y, e_z) (the paper's
// figure with their numbering is not recoverable); D3Q19 drops the eight
// corners.  With this numbering the opposite of a is Q-1-a, the property
// Sec. 2.1 designs its numbering for; a static_assert checks it.
// Weights are Qian et al. (1992) by speed class |e|^2.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace lbm {

struct D2Q9 {
    static constexpr int Q = 9, D = 2, ID = 0;
    __host__ __device__ static constexpr int e(int a, int k)
    {
        return k == 0 ? a / 3 - 1 : (k == 1 ? a % 3 - 1 : 0);
    }
    __host__ __device__ static constexpr double w(int a)
    {
        return (e(a, 0) * e(a, 0) + e(a, 1) * e(a, 1)) == 0   ? 4.0 / 9.0
               : (e(a, 0) * e(a, 0) + e(a, 1) * e(a, 1)) == 1 ? 1.0 / 9.0
                                                              : 1.0 / 36.0;
    }
    // direction number of the vector (ex, ey, ez)
    __host__ __device__ static constexpr int index_of(int ex, int ey, int ez)
    {
        return 3 * (ex + 1) + (ey + 1) + 0 * ez;
    }
};

struct D3Q27 {
    static constexpr int Q = 27, D = 3, ID = 2;
    __host__ __device__ static constexpr int e(int a, int k)
    {
        return k == 0 ? a / 9 - 1 : (k == 1 ? (a / 3) % 3 - 1 : a % 3 - 1);
    }
    __host__ __device__ static constexpr int s2(int a)
    {
        return e(a, 0) * e(a, 0) + e(a, 1) * e(a, 1) + e(a, 2) * e(a, 2);
    }
    __host__ __device__ static constexpr double w(int a)
    {
        return s2(a) == 0 ? 8.0 / 27.0 : s2(a) == 1 ? 2.0 / 27.0 : s2(a) == 2 ? 1.0 / 54.0 : 1.0 / 216.0;
    }
    __host__ __device__ static constexpr int index_of(int ex, int ey, int ez)
    {
        return 9 * (ex + 1) + 3 * (ey + 1) + (ez + 1);
    }
};

struct D3Q19 {
    static constexpr int Q = 19, D = 3, ID = 1;
    // index of the a-th non-corner vector within the 3x3x3 lexicographic cube
    __host__ __device__ static constexpr int cube(int a)
    {
        int k = 0;
        for (int c = 0; c < 27; ++c) {
            if (D3Q27::s2(c) == 3)
                continue;
            if (k == a)
                return c;
            ++k;
        }
        return -1;
    }
    __host__ __device__ static constexpr int e(int a, int k) { return D3Q27::e(cube(a), k); }
    __host__ __device__ static constexpr double w(int a)
    {
        return D3Q27::s2(cube(a)) == 0 ? 1.0 / 3.0 : D3Q27::s2(cube(a)) == 1 ? 1.0 / 18.0 : 1.0 / 36.0;
    }
    // cube index minus the corners (0, 2, 6, 8, 18, 20, 24, 26) before it
    __host__ __device__ static constexpr int index_of(int ex, int ey, int ez)
    {
        const int c = D3Q27::index_of(ex, ey, ez);
        return c - (c > 0) - (c > 2) - (c > 6) - (c > 8) - (c > 18) - (c > 20) - (c > 24);
    }
};

template <class L>
__host__ __device__ constexpr int opp(int a)
{
    return L::Q - 1 - a;
}

// The weights t_a (4/9, 1/9, 1/36; 1/3, 1/18; 8/27, 2/27, 1/54, 1/216) are
// not binary fractions, and every one of them rounds up in FP32 (by 7.45e-9
// relative, 1/3 by 2.98e-8).  So 3 sum_a t_a e_a e_a comes out as
// (1 + 7.45e-9) I instead of I on all three lattices, and every collision
// multiplies the momentum carried by the equilibrium by 1 + 7.45e-9 omega.
// Over thousands of steps that bias, not rounding noise, dominates the FP32
// velocity error (4e-5 of the flow speed after 5000 Taylor-Green steps at
// omega = 1.25).  FP32 arithmetic therefore applies the weight of the odd
// (momentum) part as two floats, t_a = hi + lo (lo the FP32 rounding of the
// residual), as fma(x, hi, x lo): one rounding of x t_a, without the bias.
template <class L>
__host__ __device__ constexpr float w_hi(int a)
{
    return float(L::w(a));
}
template <class L>
__host__ __device__ constexpr float w_lo(int a)
{
    return float(L::w(a) - double(float(L::w(a))));
}

template <class L>
constexpr bool check_set()
{
    double sw = 0.0;
    for (int a = 0; a < L::Q; ++a) {
        for (int k = 0; k < 3; ++k)
            if (L::e(opp<L>(a), k) != -L::e(a, k))
                return false;
        if (L::index_of(L::e(a, 0), L::e(a, 1), L::e(a, 2)) != a)
            return false;
        sw += L::w(a);
    }
    return sw > 1.0 - 1e-12 && sw < 1.0 + 1e-12;
}
static_assert(check_set<D2Q9>(), "D2Q9 numbering");
static_assert(check_set<D3Q19>(), "D3Q19 numbering");
static_assert(check_set<D3Q27>(), "D3Q27 numbering");

// ---- moment basis of the multiple-relaxation-time collision -----------------
// Rows orthogonal over the velocity set: the monomials e_x^i e_y^j e_z^k
// (i, j, k <= 2) by degree, |e|^2 first among degree two, orthogonalised in
// that order and scaled to coprime integers (d'Humieres et al. 2002 build
// theirs the same way).  kind: 0 density and momentum (conserved), 1 the
// bulk row (from |e|^2), 2 the traceless stress, 3 / 4 the higher rows of
// even / odd degree.  check_mrt verifies at compile time that the rows are
// pairwise orthogonal, that row 0 is 1 and rows 1..D are the velocity
// components, and the kinds' counts.
template <class L>
struct MrtBasis;
template <>
struct MrtBasis<D2Q9> {
    static constexpr signed char kind[9] = {0, 0, 0, 1, 2, 2, 4, 4, 3};
    static constexpr signed char M[9][9] = {
        {1, 1, 1, 1, 1, 1, 1, 1, 1},
        {-1, -1, -1, 0, 0, 0, 1, 1, 1},
        {-1, 0, 1, -1, 0, 1, -1, 0, 1},
        {2, -1, 2, -1, -4, -1, 2, -1, 2},
        {0, 1, 0, -1, 0, -1, 0, 1, 0},
        {1, 0, -1, 0, 0, 0, -1, 0, 1},
        {-1, 0, 1, 2, 0, -2, -1, 0, 1},
        {-1, 2, -1, 0, 0, 0, 1, -2, 1},
        {1, -2, 1, -2, 4, -2, 1, -2, 1},
    };
};
template <>
struct MrtBasis<D3Q19> {
    static constexpr signed char kind[19] = {0, 0, 0, 0, 1, 2, 2, 2, 2, 2, 4, 4, 4, 4, 4, 4, 3, 3, 3};
    static constexpr signed char M[19][19] = {
        {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
        {-1, -1, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1},
        {-1, 0, 0, 0, 1, -1, -1, -1, 0, 0, 0, 1, 1, 1, -1, 0, 0, 0, 1},
        {0, -1, 0, 1, 0, -1, 0, 1, -1, 0, 1, -1, 0, 1, 0, -1, 0, 1, 0},
        {8, 8, -11, 8, 8, 8, -11, 8, -11, -30, -11, 8, -11, 8, 8, 8, -11, 8, 8},
        {1, 1, 2, 1, 1, -2, -1, -2, -1, 0, -1, -2, -1, -2, 1, 1, 2, 1, 1},
        {1, 0, 0, 0, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, -1, 0, 0, 0, 1},
        {0, 1, 0, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, -1, 0, 1, 0},
        {1, -1, 0, -1, 1, 0, 1, 0, -1, 0, -1, 0, 1, 0, 1, -1, 0, -1, 1},
        {0, 0, 0, 0, 0, 1, 0, -1, 0, 0, 0, -1, 0, 1, 0, 0, 0, 0, 0},
        {-3, 0, 0, 0, 3, 2, 2, 2, 0, 0, 0, -2, -2, -2, -3, 0, 0, 0, 3},
        {0, -3, 0, 3, 0, 2, 0, -2, 2, 0, -2, 2, 0, -2, 0, -3, 0, 3, 0},
        {-3, 2, 2, 2, -3, 0, 0, 0, 0, 0, 0, 0, 0, 0, 3, -2, -2, -2, 3},
        {0, -1, 2, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -2, 1, 0},
        {0, 0, 0, 0, 0, -1, 0, 1, 2, 0, -2, -1, 0, 1, 0, 0, 0, 0, 0},
        {0, 0, 0, 0, 0, -1, 2, -1, 0, 0, 0, 1, -2, 1, 0, 0, 0, 0, 0},
        {5, -2, -6, -2, 5, -2, -6, -2, 8, 4, 8, -2, -6, -2, 5, -2, -6, -2, 5},
        {0, 3, -6, 3, 0, -2, 4, -2, -2, 4, -2, -2, 4, -2, 0, 3, -6, 3, 0},
        {0, 0, 0, 0, 0, 1, -2, 1, -2, 4, -2, 1, -2, 1, 0, 0, 0, 0, 0},
    };
};
template <>
struct MrtBasis<D3Q27> {
    static constexpr signed char kind[27] = {0, 0, 0, 0, 1, 2, 2, 2, 2, 2, 4, 4, 4, 4, 4, 4, 4, 3, 3, 3, 3, 3, 3, 4, 4, 4, 3};
    static constexpr signed char M[27][27] = {
        {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
        {-1, -1, -1, -1, -1, -1, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1, 1},
        {-1, -1, -1, 0, 0, 0, 1, 1, 1, -1, -1, -1, 0, 0, 0, 1, 1, 1, -1, -1, -1, 0, 0, 0, 1, 1, 1},
        {-1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1},
        {1, 0, 1, 0, -1, 0, 1, 0, 1, 0, -1, 0, -1, -2, -1, 0, -1, 0, 1, 0, 1, 0, -1, 0, 1, 0, 1},
        {0, 1, 0, 1, 2, 1, 0, 1, 0, -2, -1, -2, -1, 0, -1, -2, -1, -2, 0, 1, 0, 1, 2, 1, 0, 1, 0},
        {1, 1, 1, 0, 0, 0, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, -1, -1, -1, 0, 0, 0, 1, 1, 1},
        {1, 0, -1, 1, 0, -1, 1, 0, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, -1, 0, 1, -1, 0, 1, -1, 0, 1},
        {0, 1, 0, -1, 0, -1, 0, 1, 0, 0, 1, 0, -1, 0, -1, 0, 1, 0, 0, 1, 0, -1, 0, -1, 0, 1, 0},
        {1, 0, -1, 0, 0, 0, -1, 0, 1, 1, 0, -1, 0, 0, 0, -1, 0, 1, 1, 0, -1, 0, 0, 0, -1, 0, 1},
        {-1, -1, -1, 0, 0, 0, 1, 1, 1, 2, 2, 2, 0, 0, 0, -2, -2, -2, -1, -1, -1, 0, 0, 0, 1, 1, 1},
        {-1, 0, 1, -1, 0, 1, -1, 0, 1, 2, 0, -2, 2, 0, -2, 2, 0, -2, -1, 0, 1, -1, 0, 1, -1, 0, 1},
        {-1, -1, -1, 2, 2, 2, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, -2, -2, -2, 1, 1, 1},
        {-1, 0, 1, 0, 0, 0, 1, 0, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, -1, 0, 0, 0, -1, 0, 1},
        {-1, 2, -1, -1, 2, -1, -1, 2, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -2, 1, 1, -2, 1, 1, -2, 1},
        {-1, 0, 1, 2, 0, -2, -1, 0, 1, -1, 0, 1, 2, 0, -2, -1, 0, 1, -1, 0, 1, 2, 0, -2, -1, 0, 1},
        {-1, 2, -1, 0, 0, 0, 1, -2, 1, -1, 2, -1, 0, 0, 0, 1, -2, 1, -1, 2, -1, 0, 0, 0, 1, -2, 1},
        {1, 1, 1, -2, -2, -2, 1, 1, 1, -2, -2, -2, 4, 4, 4, -2, -2, -2, 1, 1, 1, -2, -2, -2, 1, 1, 1},
        {1, 0, -1, 0, 0, 0, -1, 0, 1, -2, 0, 2, 0, 0, 0, 2, 0, -2, 1, 0, -1, 0, 0, 0, -1, 0, 1},
        {1, -2, 1, 1, -2, 1, 1, -2, 1, -2, 4, -2, -2, 4, -2, -2, 4, -2, 1, -2, 1, 1, -2, 1, 1, -2, 1},
        {1, 0, -1, -2, 0, 2, 1, 0, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, -1, 0, 1, 2, 0, -2, -1, 0, 1},
        {1, -2, 1, 0, 0, 0, -1, 2, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, -1, 2, -1, 0, 0, 0, 1, -2, 1},
        {1, -2, 1, -2, 4, -2, 1, -2, 1, 1, -2, 1, -2, 4, -2, 1, -2, 1, 1, -2, 1, -2, 4, -2, 1, -2, 1},
        {-1, 0, 1, 2, 0, -2, -1, 0, 1, 2, 0, -2, -4, 0, 4, 2, 0, -2, -1, 0, 1, 2, 0, -2, -1, 0, 1},
        {-1, 2, -1, 0, 0, 0, 1, -2, 1, 2, -4, 2, 0, 0, 0, -2, 4, -2, -1, 2, -1, 0, 0, 0, 1, -2, 1},
        {-1, 2, -1, 2, -4, 2, -1, 2, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -2, 1, -2, 4, -2, 1, -2, 1},
        {1, -2, 1, -2, 4, -2, 1, -2, 1, -2, 4, -2, 4, -8, 4, -2, 4, -2, 1, -2, 1, -2, 4, -2, 1, -2, 1},
    };
};

template <class L>
constexpr bool check_mrt()
{
    using B = MrtBasis<L>;
    for (int a = 0; a < L::Q; ++a) {
        if (B::M[0][a] != 1)
            return false;
        for (int k = 0; k < L::D; ++k)
            if (B::M[1 + k][a] != L::e(a, k))
                return false;
    }
    int nkind[5] = {0, 0, 0, 0, 0};
    for (int r = 0; r < L::Q; ++r) {
        ++nkind[B::kind[r]];
        for (int s = r + 1; s < L::Q; ++s) {
            long dot = 0;
            for (int a = 0; a < L::Q; ++a)
                dot += (long)B::M[r][a] * B::M[s][a];
            if (dot != 0)
                return false;
        }
    }
    return nkind[0] == L::D + 1 && nkind[1] == 1 && nkind[2] == (L::D == 3 ? 5 : 2);
}
static_assert(check_mrt<D2Q9>(), "D2Q9 moment basis");
static_assert(check_mrt<D3Q19>(), "D3Q19 moment basis");
static_assert(check_mrt<D3Q27>(), "D3Q27 moment basis");

// Compile-time loop: f(std::integral_constant<int, I>) for I in [B, E).
template <int B, int E>
struct SFor {
    template <class F>
    __host__ __device__ __forceinline__ static void run(F &&f)
    {
        if constexpr (B < E) {
            f(std::integral_constant<int, B>{});
            SFor<B + 1, E>::run(f);
        }
    }
};

// ---- storage codecs -------------------------------------------------------
// Values are stored as (f_a - sigma*t_a) in T and decoded to the arithmetic
// type R.  Encoding rounds to nearest even; decoding is exact.
enum StorageId { ST_F64 = 0, ST_F32 = 1, ST_F16S = 2, ST_BF16S = 3 };

template <int S>
struct Sto;

template <>
struct Sto<ST_F64> {
    using T = double;
    using R = double;
    __device__ __forceinline__ static R dec(T v) { return v; }
    __device__ __forceinline__ static T enc(R v) { return v; }
};
template <>
struct Sto<ST_F32> {
    using T = float;
    using R = float;
    __device__ __forceinline__ static R dec(T v) { return v; }
    __device__ __forceinline__ static T enc(R v) { return v; }
};
template <>
struct Sto<ST_F16S> {
    using T = unsigned short;
    using R = float;
    __device__ __forceinline__ static R dec(T v) { return __half2float(__ushort_as_half(v)); }
    __device__ __forceinline__ static T enc(R v) { return __half_as_ushort(__float2half_rn(v)); }
};
template <>
struct Sto<ST_BF16S> {
    using T = unsigned short;
    using R = float;
    __device__ __forceinline__ static R dec(T v) { return __bfloat162float(__ushort_as_bfloat16(v)); }
    __device__ __forceinline__ static T enc(R v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
};

}  // namespace lbm
