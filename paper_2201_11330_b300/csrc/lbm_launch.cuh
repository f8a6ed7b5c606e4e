// lbm_launch.cuh -- host-side dispatch from a Launch descriptor to the
// template instantiation of each kernel (one translation unit per lattice).
#pragma once

#include "lbm_adjoint.cuh"
#include "lbm_geo.cuh"
#include "lbm_kernels.cuh"
#include "lbm_pair.cuh"

namespace lbm {

template <class F>
inline cudaError_t with_bool(bool b, F &&f)
{
    return b ? f(std::true_type{}) : f(std::false_type{});
}

template <int M>
using model_c = std::integral_constant<int, M>;

// One instantiation per collision model (Model).  PART 0: every model but
// MRT; PART 1: MRT only (FP64 / FP32 storage; the host refuses the rest).  The
// MRT kernels are instantiated in translation units of their own
// (lbm_<lattice>_<storage>_mrt.cu), which compile in parallel with the rest.
template <int S, int PART, class F>
inline cudaError_t with_model(int m, F &&f)
{
    if constexpr (PART == 1) {
        if constexpr (S == ST_F64 || S == ST_F32) {
            if (m == M_MRT)
                return f(model_c<M_MRT>{});
        }
        return cudaErrorInvalidValue;
    } else {
        switch (m) {
        case M_INC:
            return f(model_c<M_INC>{});
        case M_COMP:
            return f(model_c<M_COMP>{});
        case M_TRT:
            return f(model_c<M_TRT>{});
        default:
            return cudaErrorInvalidValue;
        }
    }
}

// The step and initialisation launches of the MRT model (PART 1 of
// launch_storage), defined in lbm_<lattice>_<storage>_mrt.cu.
template <class L, int S>
cudaError_t launch_mrt(const Launch &l);

// plain D3Q27 pull / gather kernels with 16-bit storage: blocks per SM bound
template <class L, int S>
constexpr int kPlainMinBlocks = (L::Q == 27 && (S == ST_F16S || S == ST_BF16S)) ? 5 : 0;
// the AA gather half also with FP32 storage (three blocks: unbounded it takes
// 97 registers, two blocks per SM)
template <class L, int S>
constexpr int kPlainGatherMinBlocks = kPlainMinBlocks<L, S> > 0 ? kPlainMinBlocks<L, S>
                                      : (L::Q == 27 && S == ST_F32) ? 3
                                                                    : 0;

// MRT step kernels: blocks per SM bound per pattern (0: the thread bound alone).
// FP32 storage, measured at 512^3 (D3Q19) and 384^3 (D3Q27), ms per launch,
// unbounded / bounded: D3Q19 at five (64 -> 48 registers, 32-72 B spilled)
// pull 4.03 / 3.53, gather 4.69 / 4.32, local 3.43 / 3.49; D3Q27 at four
// (80 -> 64 registers) pull 2.67 / 2.71, gather 3.40 / 2.96, local 2.62 /
// 2.52.  One block more per SM was slower on every pattern.
template <class L, int S, int PAT>
constexpr int kMrtMinBlocks = S != ST_F32   ? 0
                              : L::Q == 19 ? (PAT == PAT_LOCAL ? 0 : 5)
                              : L::Q == 27 ? (PAT == PAT_PULL ? 0 : 4)
                                           : 0;

template <class L, int S, int PART = 0>
cudaError_t launch_storage(const Launch &l)
{
    using T = typename Sto<S>::T;
    const T *src = (const T *)l.src;
    T *dst = (T *)l.dst;
    if constexpr (PART == 0 && (S == ST_F64 || S == ST_F32)) {
        if ((l.kind == K_STEP || l.kind == K_INIT) && l.model == M_MRT)
            return launch_mrt<L, S>(l);
    }
    if (l.kind == K_STEP && l.pair && !l.skip) {
        if constexpr (S == ST_F16S || S == ST_BF16S) {
            const dim3 grid((l.sp.nx + 2 * kPairThreads - 1) / (2 * kPairThreads), l.sp.ny, l.sp.nz);
            return with_model<S, PART>(l.model, [&](auto C) {
                return with_bool(l.force, [&](auto Fo) {
                    constexpr int c = decltype(C)::value;
                    constexpr bool fo = decltype(Fo)::value;
                    const auto *s16 = (const unsigned short *)l.src;
                    auto *d16 = (unsigned short *)l.dst;
                    return with_bool(l.sp.partials != nullptr, [&](auto Rd) {
                        constexpr bool rd = decltype(Rd)::value;
                        // blocks per SM of each paired kernel (0: unbounded),
                        // measured on B300 (512^3 D3Q19, 768^3 D3Q27 cavities)
                        constexpr int mb_pull = L::Q == 27 ? 7 : L::Q == 19 ? 8 : 0;
                        constexpr int mb_gather = L::Q == 27 ? 6 : L::Q == 19 ? 8 : 0;
                        constexpr int mb_local = L::Q == 19 ? 8 : 0;
                        auto go = [&](auto P, auto MB) {
                            constexpr int pt = decltype(P)::value, m = decltype(MB)::value;
                            if constexpr (m > 0 && !rd)
                                k_step_pair_bounded<L, S, pt, c, fo, m>
                                    <<<grid, kPairThreads, 0, l.stream>>>(s16, d16, l.sp);
                            else
                                k_step_pair<L, S, pt, c, fo, rd>
                                    <<<grid, kPairThreads, 0, l.stream>>>(s16, d16, l.sp);
                        };
                        using std::integral_constant;
                        if (l.pattern == PAT_PULL)
                            go(integral_constant<int, PAT_PULL>{}, integral_constant<int, mb_pull>{});
                        else if (l.pattern == PAT_GATHER)
                            go(integral_constant<int, PAT_GATHER>{},
                               integral_constant<int, mb_gather>{});
                        else
                            go(integral_constant<int, PAT_LOCAL>{}, integral_constant<int, mb_local>{});
                        return cudaGetLastError();
                    });
                });
            });
        } else {
            return cudaErrorInvalidValue;
        }
    }
    if (l.kind == K_STEP && l.geo) {
        return with_model<S, PART>(l.model, [&](auto C) {
            return with_bool(l.force, [&](auto Fo) {
                constexpr int c = decltype(C)::value;
                constexpr bool fo = decltype(Fo)::value;
                auto go = [&](auto Mo) {
                    constexpr int mo = decltype(Mo)::value;
                    if constexpr (S == ST_F64)  // FP64-ALU bound: unbounded
                        k_step_geo<L, S, c, fo, mo><<<l.grid, l.block, 0, l.stream>>>(src, dst,
                                                                                    l.sp);
                    else
                        k_step_geo_bounded<L, S, c, fo, mo>
                            <<<l.grid, l.block, 0, l.stream>>>(src, dst, l.sp);
                };
                if (l.mon == 1)
                    go(std::integral_constant<int, 1>{});
                else if (l.mon == 2)
                    go(std::integral_constant<int, 2>{});
                else
                    go(std::integral_constant<int, 0>{});
                return cudaGetLastError();
            });
        });
    }
    if (l.kind == K_STEP && l.skip) {
        return with_model<S, PART>(l.model, [&](auto C) {
            return with_bool(l.force, [&](auto Fo) {
                constexpr int c = decltype(C)::value;
                constexpr bool fo = decltype(Fo)::value;
                if constexpr (S == ST_F16S || S == ST_BF16S) {
                    if (l.pair) {
                        const auto *s16 = (const unsigned short *)l.src;
                        auto *d16 = (unsigned short *)l.dst;
                        if (l.mon == 1)
                            k_step_pair_skip<L, S, c, fo, 1>
                                <<<l.grid, kPairThreads, 0, l.stream>>>(s16, d16, l.sp);
                        else if (l.mon == 2)
                            k_step_pair_skip<L, S, c, fo, 2>
                                <<<l.grid, kPairThreads, 0, l.stream>>>(s16, d16, l.sp);
                        else
                            k_step_pair_skip<L, S, c, fo, 0>
                                <<<l.grid, kPairThreads, 0, l.stream>>>(s16, d16, l.sp);
                        return cudaGetLastError();
                    }
                }
                if (l.mon == 1)
                    k_step_skip<L, S, c, fo, 1><<<l.grid, l.block, 0, l.stream>>>(src, dst, l.sp);
                else if (l.mon == 2)
                    k_step_skip<L, S, c, fo, 2><<<l.grid, l.block, 0, l.stream>>>(src, dst, l.sp);
                else
                    k_step_skip<L, S, c, fo, 0><<<l.grid, l.block, 0, l.stream>>>(src, dst, l.sp);
                return cudaGetLastError();
            });
        });
    }
    if constexpr (PART == 0) {  // model-independent kernels: not in the MRT units
        if (l.kind == K_FLAGS) {
            if constexpr (S == ST_F32) {  // storage-independent: one instantiation per lattice
                k_node_flags<L><<<l.grid, l.block, 0, l.stream>>>(l.flags, l.sp, l.pair);
                return cudaGetLastError();
            } else {
                return cudaErrorInvalidValue;
            }
        }
        if (l.kind == K_LINKS) {
            if constexpr (S == ST_F32) {  // storage-independent: one instantiation per lattice
                k_links<L><<<l.grid, l.block, 0, l.stream>>>(l.solid, l.links, l.nsolid, l.sp);
                return cudaGetLastError();
            } else {
                return cudaErrorInvalidValue;
            }
        }
    }
    if (l.kind == K_STEP) {
        if (l.pattern == PAT_PULL) {
            if constexpr (PART == 0) {
                if (l.uout) {
                    // adjoint recompute: incompressible BGK only
                    return with_bool(l.force, [&](auto Fo) {
                        k_step<L, S, PAT_PULL, M_INC, decltype(Fo)::value, true>
                            <<<l.grid, l.block, 0, l.stream>>>(src, dst, l.sp);
                        return cudaGetLastError();
                    });
                }
            }
            return with_model<S, PART>(l.model, [&](auto C) {
                return with_bool(l.force, [&](auto Fo) {
                    return with_bool(l.sp.partials != nullptr, [&](auto Rd) {
                        constexpr int c = decltype(C)::value;
                        constexpr bool fo = decltype(Fo)::value, rd = decltype(Rd)::value;
                        constexpr int mrt_mb = c == M_MRT ? kMrtMinBlocks<L, S, PAT_PULL> : 0;
                        if constexpr (mrt_mb > 0 && !rd)
                            k_step_bounded<L, S, PAT_PULL, c, fo, mrt_mb>
                                <<<l.grid, l.block, 0, l.stream>>>(src, dst, l.sp);
                        else if constexpr (kPlainMinBlocks<L, S> > 0 && !rd)
                            k_step_bounded<L, S, PAT_PULL, c, fo, kPlainMinBlocks<L, S>>
                                <<<l.grid, l.block, 0, l.stream>>>(src, dst, l.sp);
                        else
                            k_step<L, S, PAT_PULL, c, fo, false, rd>
                                <<<l.grid, l.block, 0, l.stream>>>(src, dst, l.sp);
                        return cudaGetLastError();
                    });
                });
            });
        }
        if (l.pattern == PAT_GATHER) {
            return with_model<S, PART>(l.model, [&](auto C) {
                return with_bool(l.force, [&](auto Fo) {
                    constexpr int c = decltype(C)::value;
                    constexpr bool fo = decltype(Fo)::value;
                    constexpr int mrt_mb = c == M_MRT ? kMrtMinBlocks<L, S, PAT_GATHER> : 0;
                    if (l.sp.partials != nullptr)
                        k_step_gather_red<L, S, c, fo><<<l.grid, l.block, 0, l.stream>>>(src, dst,
                                                                                         l.sp);
                    else if constexpr (mrt_mb > 0)
                        k_step_bounded<L, S, PAT_GATHER, c, fo, mrt_mb>
                            <<<l.grid, l.block, 0, l.stream>>>(src, dst, l.sp);
                    else if constexpr (kPlainGatherMinBlocks<L, S> > 0)
                        k_step_bounded<L, S, PAT_GATHER, c, fo, kPlainGatherMinBlocks<L, S>>
                            <<<l.grid, l.block, 0, l.stream>>>(src, dst, l.sp);
                    else
                        k_step<L, S, PAT_GATHER, c, fo, false, false>
                            <<<l.grid, l.block, 0, l.stream>>>(src, dst, l.sp);
                    return cudaGetLastError();
                });
            });
        }
        return with_model<S, PART>(l.model, [&](auto C) {
            return with_bool(l.force, [&](auto Fo) {
                return with_bool(l.sp.partials != nullptr, [&](auto Rd) {
                    constexpr int c = decltype(C)::value;
                    constexpr bool fo = decltype(Fo)::value, rd = decltype(Rd)::value;
                    constexpr int mrt_mb = c == M_MRT ? kMrtMinBlocks<L, S, PAT_LOCAL> : 0;
                    if constexpr (mrt_mb > 0 && !rd)
                        k_step_bounded<L, S, PAT_LOCAL, c, fo, mrt_mb>
                            <<<l.grid, l.block, 0, l.stream>>>(src, dst, l.sp);
                    else
                        k_step<L, S, PAT_LOCAL, c, fo, false, rd>
                            <<<l.grid, l.block, 0, l.stream>>>(src, dst, l.sp);
                    return cudaGetLastError();
                });
            });
        });
    }
    if (l.kind == K_INIT) {
        return with_bool(l.pattern == 1, [&](auto AA) {
            return with_model<S, PART>(l.model, [&](auto C) {
                return with_bool(l.force, [&](auto Fo) {
                    constexpr bool aa = decltype(AA)::value, fo = decltype(Fo)::value;
                    constexpr int c = decltype(C)::value;
                    if (l.in_f32)
                        k_init<L, S, aa, c, fo, float><<<l.grid, l.block, 0, l.stream>>>(
                            dst, l.sp, (const float *)l.p0, (const float *)l.u0);
                    else
                        k_init<L, S, aa, c, fo, double><<<l.grid, l.block, 0, l.stream>>>(
                            dst, l.sp, (const double *)l.p0, (const double *)l.u0);
                    return cudaGetLastError();
                });
            });
        });
    }
    if constexpr (PART == 0) {  // the adjoint and the moments: not in the MRT units
        if (l.kind == K_ADJ) {
            using R = typename Sto<S>::R;
            return with_bool(l.force, [&](auto Fo) {
                constexpr bool fo = decltype(Fo)::value;
                if constexpr (std::is_same<R, float>::value && fo && L::Q == 19)
                    k_adjoint_bounded<L, R, fo, 5><<<l.grid, l.block, 0, l.stream>>>(l.sp, l.ap);
                else
                    k_adjoint<L, R, fo><<<l.grid, l.block, 0, l.stream>>>(l.sp, l.ap);
                return cudaGetLastError();
            });
        }
        if (l.kind == K_SEED) {
            return with_bool(l.force, [&](auto Fo) {
                k_adjoint_seed<L, S, decltype(Fo)::value><<<l.grid, l.block, 0, l.stream>>>(l.sp, l.ap);
                return cudaGetLastError();
            });
        }
        if (l.kind == K_FLUSH) {
            using R = typename Sto<S>::R;
            k_adjoint_flush<R><<<l.grid, l.block, 0, l.stream>>>((R *)l.ap.gF, l.ap.dJdF, l.count);
            return cudaGetLastError();
        }
        if (l.kind == K_MOMENTS) {
            return with_bool(l.comp, [&](auto C) {
                return with_bool(l.force, [&](auto Fo) {
                    constexpr bool c = decltype(C)::value, fo = decltype(Fo)::value;
                    if constexpr (S == ST_F16S || S == ST_BF16S) {
                        // 16-bit storage, the node's own slots: two nodes per
                        // thread, one 32-bit load per slot
                        if (l.pattern != FORM_STREAMED && l.sp.nx % 2 == 0) {
                            MomParams mp = l.mp;
                            mp.xseg = (l.sp.nx + 2 * kPairThreads - 1) / (2 * kPairThreads);
                            mp.nseg = mp.xseg * l.sp.ny * l.sp.nz;
                            const auto *s16 = (const unsigned short *)l.src;
                            if (l.pattern == FORM_LOCAL)
                                k_moments_pair<L, S, FORM_LOCAL, c, fo>
                                    <<<l.grid, kPairThreads, 0, l.stream>>>(s16, l.sp, mp);
                            else
                                k_moments_pair<L, S, FORM_SWAPPED, c, fo>
                                    <<<l.grid, kPairThreads, 0, l.stream>>>(s16, l.sp, mp);
                            return cudaGetLastError();
                        }
                    }
                    switch (l.pattern) {
                    case FORM_LOCAL:
                        k_moments<L, S, FORM_LOCAL, c, fo><<<l.grid, l.block, 0, l.stream>>>(src, l.sp, l.mp);
                        break;
                    case FORM_SWAPPED:
                        k_moments<L, S, FORM_SWAPPED, c, fo><<<l.grid, l.block, 0, l.stream>>>(src, l.sp, l.mp);
                        break;
                    default:
                        k_moments<L, S, FORM_STREAMED, c, fo><<<l.grid, l.block, 0, l.stream>>>(src, l.sp, l.mp);
                        break;
                    }
                    return cudaGetLastError();
                });
            });
        }
    }
    return cudaErrorInvalidValue;
}



template <class L, int S>
cudaError_t launch_mrt(const Launch &l)
{
    return launch_storage<L, S, 1>(l);
}

}  // namespace lbm
