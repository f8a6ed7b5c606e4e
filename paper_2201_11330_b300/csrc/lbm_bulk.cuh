// lbm_bulk.cuh -- the fused step with its loads staged through shared memory
// by bulk asynchronous copies (cp.async.bulk, completion on an mbarrier).
//
// Same arithmetic as k_step (lbm_kernels.cuh), different data movement: a
// persistent block walks segments of kBulkSeg nodes along x.  For every
// direction a, one elected thread copies the whole source row segment (the
// row (y - e_ay, z - e_az) of slot a or abar, plus a 16-byte halo on each
// side for the x shift) from HBM into a shared-memory stage with one bulk
// copy; kBulkStages segments are in flight per block, so the copy engine,
// not registers, holds the bytes in flight.  Threads then read their Q
// values from shared memory, collide, and store straight to HBM.
//
// Preconditions checked by the host: nx and N multiples of 16/sizeof(T)
// (every copy starts and ends on a 16-byte boundary), workspace 256-aligned.
// Every wait is bounded: on time-out the block records an error word, drains
// its own copies (bounded) and leaves.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

constexpr int kBulkSeg = 256;  // nodes per segment = threads per block
constexpr int kBulkStages = 3;
constexpr unsigned kWaitLimit = 1u << 24;  // try_wait polls before giving up

struct BulkParams {
    int nseg;       // xseg * ny * nz
    int xseg;       // segments per row
    unsigned *err;  // set non-zero when a wait timed out
};

template <class T>
__host__ __device__ constexpr int bulk_halo()
{
    return 16 / (int)sizeof(T);
}
template <class T>
__host__ __device__ constexpr int bulk_row()
{
    return kBulkSeg + 2 * bulk_halo<T>();
}
template <class L, class T>
__host__ __device__ constexpr size_t bulk_smem_bytes()
{
    return (size_t)kBulkStages * L::Q * bulk_row<T>() * sizeof(T) + kBulkStages * sizeof(uint64_t);
}

// ---- PTX wrappers -------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity)
{
    for (unsigned i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(bar, parity))
            return true;
    return false;
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes,
                                              uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- where direction a's incoming populations of row (y, z) come from --------
// row: row index (y' + ny z') of the source row; slot: slot to read; yzwall:
// the link crosses a y or z wall, so the population is the node's own bounce
// slot, read without x shift.
template <class L, int PAT, int a>
__device__ __forceinline__ void row_source(const StepParams &p, int y, int z, int &row, int &slot,
                                           bool &yzwall)
{
    constexpr int ey = L::e(a, 1), ez = L::e(a, 2);
    constexpr int b = opp<L>(a);
    yzwall = false;
    if constexpr (PAT == PAT_LOCAL) {
        row = y + p.ny * z;
        slot = a;
        return;
    }
    int ys = y - ey, zs = z - ez;
    if (ys < 0 || ys >= p.ny) {
        if (p.periodic & 2)
            ys = ys < 0 ? ys + p.ny : ys - p.ny;
        else
            yzwall = true;
    }
    if (zs < 0 || zs >= p.nz) {
        if (p.periodic & 4)
            zs = zs < 0 ? zs + p.nz : zs - p.nz;
        else
            yzwall = true;
    }
    if (yzwall) {
        row = y + p.ny * z;
        slot = (PAT == PAT_PULL) ? b : a;
    } else {
        row = ys + p.ny * zs;
        slot = (PAT == PAT_PULL) ? a : b;
    }
}

template <int PAT>
__device__ __forceinline__ void seg_range(int x0, int nx, int H, int &lo, int &hi)
{
    if (PAT == PAT_LOCAL) {
        lo = x0;
        hi = min(x0 + kBulkSeg, nx);
    } else {
        lo = max(x0 - H, 0);
        hi = min(x0 + kBulkSeg + H, nx);
    }
}

// Thread 0: copy segment `seg` (all Q source rows) into stage buffer sb.
template <class L, int S, int PAT>
__device__ __forceinline__ void bulk_issue(const typename Sto<S>::T *src, typename Sto<S>::T *sb,
                                           uint64_t *bar, const StepParams &p, int seg, int xseg)
{
    using T = typename Sto<S>::T;
    constexpr int H = bulk_halo<T>(), ROW = bulk_row<T>();
    const int xs = seg % xseg, r = seg / xseg;
    const int y = r % p.ny, z = r / p.ny, x0 = xs * kBulkSeg;
    int lo, hi;
    seg_range<PAT>(x0, p.nx, H, lo, hi);
    const unsigned bytes = (unsigned)((hi - lo) * (int)sizeof(T));
    mbar_expect_tx(bar, bytes * L::Q);
    const size_t N = (size_t)p.N;
    SFor<0, L::Q>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        int row, slot;
        bool yzw;
        row_source<L, PAT, a>(p, y, z, row, slot, yzw);
        const T *g = src + (size_t)slot * N + (size_t)row * p.nx + lo;
        T *d = sb + a * ROW + (lo - (x0 - H));
        bulk_copy_g2s(d, g, bytes, bar);
    });
}

// One node of a staged segment.  IROW: the row is interior in y and z.
template <class L, int S, int PAT, int MODEL, bool FORCE, bool IROW>
__device__ __forceinline__ void bulk_node(const typename Sto<S>::T *src, typename Sto<S>::T *dst,
                                          typename Sto<S>::T *sb, const StepParams &p, int x0,
                                          int y, int z, int tid)
{
    using T = typename Sto<S>::T;
    using R = typename Sto<S>::R;
    constexpr int Q = L::Q, H = bulk_halo<T>(), ROW = bulk_row<T>();
    const Coef<R> &c = coef<R>(p);
    const size_t N = (size_t)p.N;
    const int x = x0 + tid;
    const int n = x + p.nx * (y + p.ny * z);
    const bool top = p.lid_on && (y == p.ny - 1);

    if constexpr (PAT != PAT_LOCAL) {
        // The halo entries at x0-1 / x0+kBulkSeg are read only by the node at
        // x = x0 / x0+kBulkSeg-1.  At the ends of the row they lie outside
        // the box: that node fills them itself (periodic wrap or bounce-back).
        if (x == 0 || x == p.nx - 1) {
            SFor<0, Q>::run([&](auto A_) {
                constexpr int a = decltype(A_)::value;
                constexpr int ex = L::e(a, 0), b = opp<L>(a);
                if constexpr (ex != 0) {
                    if ((ex == 1 && x == 0) || (ex == -1 && x == p.nx - 1)) {
                        int row, slot;
                        bool yzw;
                        row_source<L, PAT, a>(p, y, z, row, slot, yzw);
                        if (!yzw) {
                            T v;
                            if (p.periodic & 1)
                                v = src[(size_t)slot * N + (size_t)row * p.nx + (ex == 1 ? p.nx - 1 : 0)];
                            else
                                v = src[(size_t)(PAT == PAT_PULL ? b : a) * N + n];
                            sb[a * ROW + H + tid - ex] = v;
                        }
                    }
                }
            });
        }
    }

    R g[Q];
    SFor<0, Q>::run([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        constexpr int ex = (PAT == PAT_LOCAL) ? 0 : L::e(a, 0);
        int sh = ex;
        if constexpr (!IROW && PAT != PAT_LOCAL) {
            int row, slot;
            bool yzw;
            row_source<L, PAT, a>(p, y, z, row, slot, yzw);
            sh = yzw ? 0 : ex;
        }
        R v = Sto<S>::dec(sb[a * ROW + H + tid - sh]);
        if constexpr (L::e(a, 1) == -1 && !IROW) {
            if (top)
                v += c.lid[a];
        }
        g[a] = v;
    });
    R F[3] = {R(0), R(0), R(0)};
    if constexpr (FORCE) {
        SFor<0, L::D>::run([&](auto K_) {
            constexpr int k = decltype(K_)::value;
            F[k] = R(p.F[k * N + n]);
        });
    }
    R u[3], s_, rho_;
    collide<L, R, MODEL, FORCE>(g, F, c, u, s_, rho_);
    if constexpr (PAT == PAT_PULL) {
        SFor<0, Q>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            st(dst + a * N + n, Sto<S>::enc(g[a]));
        });
    } else if constexpr (PAT == PAT_LOCAL) {
        SFor<0, Q>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            st(dst + opp<L>(a) * N + n, Sto<S>::enc(g[a]));
        });
    } else {
        AxisNbr X, Y, Z;
        make_axes<L, IROW>(p, x, y, z, X, Y, Z);
        SFor<0, Q>::run([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            constexpr int b = opp<L>(a);
            int off;
            bool wall;
            upstream<L, b>(X, Y, Z, off, wall);  // x + e_a
            T *ptr = wall ? dst + b * N + n : dst + a * N + (n + off);
            st(ptr, Sto<S>::enc(g[a]));
        });
    }
}

template <class L, int S, int PAT, int MODEL, bool FORCE>
__global__ void __launch_bounds__(kBulkSeg) k_step_bulk(const typename Sto<S>::T *src,
                                                        typename Sto<S>::T *dst, const StepParams p,
                                                        const BulkParams bp)
{
    using T = typename Sto<S>::T;
    constexpr int Q = L::Q, ROW = bulk_row<T>();
    extern __shared__ __align__(128) unsigned char smem[];
    T *bufs = (T *)smem;
    uint64_t *bars = (uint64_t *)(smem + (size_t)kBulkStages * Q * ROW * sizeof(T));
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < kBulkStages; ++s)
            mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < kBulkStages; ++k) {
            const int seg = blockIdx.x + k * gridDim.x;
            if (seg < bp.nseg)
                bulk_issue<L, S, PAT>(src, bufs + k * Q * ROW, &bars[k], p, seg, bp.xseg);
        }
    }
    for (int k = 0;; ++k) {
        const int seg = blockIdx.x + k * gridDim.x;
        if (seg >= bp.nseg)
            break;
        const int s = k % kBulkStages;
        const unsigned parity = (unsigned)(k / kBulkStages) & 1u;
        const bool ok = mbar_wait_bounded(&bars[s], parity);
        if (__syncthreads_or(!ok)) {
            // a copy never completed: record it, wait (bounded) for this
            // block's outstanding copies, and leave
            if (tid == 0) {
                atomicOr(bp.err, 1u);
                for (int j = k; j < k + kBulkStages; ++j) {
                    if (blockIdx.x + j * gridDim.x >= bp.nseg)
                        break;
                    mbar_wait_bounded(&bars[j % kBulkStages], (unsigned)(j / kBulkStages) & 1u);
                }
            }
            return;
        }
        T *sb = bufs + s * Q * ROW;
        const int xs = seg % bp.xseg, r = seg / bp.xseg;
        const int y = r % p.ny, z = r / p.ny, x0 = xs * kBulkSeg;
        if (x0 + tid < p.nx) {
            const bool irow = y > 0 && y < p.ny - 1 && (L::D == 2 || (z > 0 && z < p.nz - 1));
            if (irow)
                bulk_node<L, S, PAT, MODEL, FORCE, true>(src, dst, sb, p, x0, y, z, tid);
            else
                bulk_node<L, S, PAT, MODEL, FORCE, false>(src, dst, sb, p, x0, y, z, tid);
        }
        __syncthreads();  // every read of stage s is done
        if (tid == 0) {
            const int nxt = blockIdx.x + (k + kBulkStages) * gridDim.x;
            if (nxt < bp.nseg) {
                fence_proxy_async_smem();
                bulk_issue<L, S, PAT>(src, sb, &bars[s], p, nxt, bp.xseg);
            }
        }
    }
}

}  // namespace lbm
