// Isotropic sweep: one leapfrog step (Eq. 3) of v^2 (d_xx + d_yy + d_zz) u with
// the order-2R central stencil of Eq. 4 on every axis, the Cerjan damping layer,
// the Ricker source and the receiver lattice fused in.
//
// Design (2.5D plane sweep after the shared-memory x-y tile plus z register
// queue of Sec. 3, rebuilt for sm_103a as a warp-specialised TMA pipeline):
//   * a CTA owns a TX x TY column of the grid and a chunk of z planes, swept
//     upward (at radius 8 the odd chunks downward);
//   * one producer warp issues TMA 3D tile loads into two shared-memory rings:
//     ring A holds plane k of u^n with an R-cell x-y halo (loads outside the
//     grid return zeros: the zero halo of Sec. 1 at no cost), ring B holds the
//     TX x TY tiles of u^{n-1} and kappa of plane k and of u^n of plane k + R.
//     Each slot has a "full" mbarrier (TMA transaction count) and an "empty"
//     mbarrier (one arrival per consumer warp), so consumer warps never wait
//     for each other and the producer runs up to LA planes ahead;
//   * each consumer thread owns 4 consecutive x points (one float4) of one row
//     and keeps their 2R+1 z neighbours in registers (plane k + R enters from
//     ring B); x and y neighbours come from the staged plane (x as 1 + R/2
//     aligned float4 reads, y as 2R).  32 x 32 tiles (the default at radius 4
//     and 8) keep the z neighbours in tensor memory instead, and each thread
//     takes two adjacent rows, which share their y reads;
//   * u^{n+1} is written in place over u^{n-1} with 128-bit evict-first stores
//     (each point's older value was staged before any thread writes it);
//   * the damping is applied in its deferred form G (2u - G u_prev + kappa Lu + s),
//     which equals multiplying both new levels by G after each step (Cerjan)
//     without rewriting u^n.
//   * a consumer fences its plain reads of a slot (fence.proxy.async) before its
//     warp releases the slot: the producer's next copy into it goes through the
//     async proxy, which the release alone does not order after those reads;
//   * consecutive single-shot steps are launched as programmatic dependents:
//     a CTA sets up its barriers (and tensor memory) before it waits for the
//     previous step, then takes its time index.
// Compulsory HBM traffic: 16 bytes per point update (read u^n, u^{n-1}, kappa;
// write u^{n+1}).  All waits are bounded (about 1 s); a CTA that gives up sets
// an error flag, drains its copies in flight and exits.
#include <atomic>

#include "fd_internal.h"
#include "launch_shape.h"
#include "ptx.cuh"
#include "rec_slot.cuh"
#include "tmem.cuh"

namespace fdk {

// ~1 s at the GB300's 2 GHz SM clock: far beyond any TMA latency.
constexpr long long kWaitLimit = 2000000000LL;

// NBT: tiles per ring B slot (u^{n-1} and kappa; z, kappa and the gradient
// for the gradient sweep).
template <int R, int TX, int TY, int LA, int NBT = 2>
struct IsoCfg {
    static constexpr int NTX = TX / 4;              // consumer threads per tile row
    // 32 x 32 tiles (radius 4 and 8; the forward and adjoint sweeps, not the
    // gradient sweep) keep their z queues in tensor memory, which frees the
    // registers for two tile rows per thread: the rows share their y-neighbour
    // reads.
    static constexpr bool TQ = ((R == 8 || R == 4) && TX == 32 && TY == 32 && NBT == 2);
    static constexpr int QS = 2 * R;                // queue ring slots per row
    static constexpr int QC = 4 * QS;               // tensor-memory columns per row
    static constexpr int RPT = TQ ? 2 : 1;          // tile rows per consumer thread
    static constexpr int NC = NTX * TY / RPT;       // consumer threads
    static constexpr int NCW = NC / 32;             // consumer warps
    static constexpr int NT = NC + 32;              // + one producer warp
    static constexpr int SW = TX + 2 * R;           // staged row width (floats)
    static constexpr int SH = TY + 2 * R;           // staged rows
    static constexpr int SLOT_A = SW * SH;          // floats per u^n plane
    // Each plane's own values for the z queue arrive as one more ring B tile
    // (u^n of plane k + R), so ring A holds only the LA + 1 planes in flight
    // rather than R planes ahead: small enough for three radius-8 or four
    // radius-4 CTAs of 160 threads per SM in the register form.
    static constexpr int NBT_ALL = NBT + 1;
    static constexpr int SLOT_B = NBT_ALL * TX * TY;   // floats per ring B plane
    static constexpr int NA = LA + 1;               // ring A slots
    // CTAs per SM the registers are budgeted for
    static constexpr int MINB = TQ ? ((R == 4 && LA == 2) ? 4 : 3) : (NT <= 160 ? (R >= 8 ? 3 : 4) : 2);
    // Tensor memory per CTA: two rows x 4 QS columns (radius 8: 128, radius 4:
    // 64).  Shared memory keeps at most three radius-8 CTAs (65 KB each) or four
    // radius-4 ones (55 KB at lookahead 2, 74 KB at 3) on an SM, so their
    // allocations (at most 384 of the 512 columns; any mix with the VTI sweep's
    // 128-column CTAs of 112 KB stays below 450) never wait.
    static constexpr int TMEM_COLS = 2 * QC;
    static constexpr int SMEM_FLOOR = 0;
    static constexpr int NB = LA + 1;               // ring B slots
    static constexpr int OFF_B = NA * SLOT_A * 4;
    static constexpr int OFF_BAR = OFF_B + NB * SLOT_B * 4;
    static constexpr int OFF_GZ = OFF_BAR + 8 * (2 * NA + 2 * NB) + 32;
    // + 4 bytes per plane of the chunk (damping factors along z), added at launch
    static constexpr int SMEM = OFF_GZ;
    static_assert(TX % 4 == 0 && R % 4 == 0, "x alignment");
    static_assert(NC % 32 == 0, "whole consumer warps");
    static_assert(!TQ || NC == 128, "tensor-memory queues: one consumer warp per lane quarter");
    static_assert((SLOT_A * 4) % 128 == 0 && (SLOT_B * 4) % 128 == 0, "slot alignment");
    static_assert(SW <= 256 && SH <= 256, "TMA box limit");
};

// The time index n of a shot: thread 0 reads it and counts this CTA; the last
// of the shot's ncta CTAs advances it (so graph replays need no per-step
// arguments).  Returns -1 to every thread when n >= n_end (a finished shot in a
// batch: its CTAs do nothing).
// step_take is the part of one thread; step_prologue shares its result with the CTA.
// With hold the time index is only read (a part of a step that another part completes).
__device__ __forceinline__ int step_take(DevState *st, unsigned ncta, int n_end, bool hold = false)
{
    int n = *reinterpret_cast<volatile int *>(&st->step);
    if (n >= n_end) return -1;
    if (hold) return n;
    __threadfence();
    if (atomicAdd(&st->done, 1u) == ncta - 1) {
        st->done = 0;
        *reinterpret_cast<volatile int *>(&st->step) = n + 1;
        __threadfence();
    }
    return n;
}

__device__ __forceinline__ int step_prologue(DevState *st, unsigned ncta, int n_end, int *sh_n)
{
    if (threadIdx.x == 0) *sh_n = step_take(st, ncta, n_end);
    __syncthreads();
    return *sh_n;
}

// The update of one thread's 4 points of plane k in row gyi (Eq. 3 with the
// damping in its deferred form, G = gx * gy * gz), with the source, the
// injection lattice (INJ) and the receivers; u^{n+1} is written over u^{n-1}.
// acc holds L u^n (the stencil sum), cu u^n, pv u^{n-1}, kv kappa, g4 the x
// damping factors and gyz = gy * gz.
template <bool INJ>
__device__ __forceinline__ void update_row(const IsoArgs &a, float *prev, const int n, const int k, const int gxi,
                                           const int gyi, const long long rowoff, const float (&acc)[4],
                                           const float (&cu)[4], const float4 pv, const float4 kv, const float4 g4,
                                           const float gyz)
{
    const float pu[4] = {pv.x, pv.y, pv.z, pv.w};
    const float ku[4] = {kv.x, kv.y, kv.z, kv.w};
    const float gu[4] = {g4.x, g4.y, g4.z, g4.w};
    float o[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float G = gu[e] * gyz;
        o[e] = fmaf(ku[e], acc[e], fmaf(2.f, cu[e], -G * pu[e]));
    }
    if (k == a.src.sz && gyi == a.src.sy && a.src.sx >= gxi && a.src.sx < gxi + 4 && n < a.src.len) {
        // constant indices only: an index computed at run time would put o in
        // local memory, stored on every update
        const float sv = a.src.tab[n];
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (a.src.sx == gxi + e) o[e] += sv;
    }
    if (INJ && k == a.inj.rk) {
        // lattice of additive sources (the adjoint's receiver residuals)
        const int ry = gyi - a.inj.ry0;
        const int row = n - a.inj.t0;
        if (ry >= 0 && ry % a.inj.rsy == 0 && ry / a.inj.rsy < a.inj.rny && row >= 0 && row < a.inj.cap) {
            const float *irow = a.inj.trace + (long long)row * a.inj.nrec + (long long)(ry / a.inj.rsy) * a.inj.rnx;
            for (int e = 0; e < 4; ++e) {
                const int rx = gxi + e - a.inj.rx0;
                if (gxi + e < a.nx && rx >= 0 && rx % a.inj.rsx == 0 && rx / a.inj.rsx < a.inj.rnx)
                    o[e] += irow[rx / a.inj.rsx];
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) o[e] *= gu[e] * gyz;

    float *dst = prev + k * a.plane + rowoff;
    if (gxi + 3 < a.nx) {
        st_cs(dst, make_float4(o[0], o[1], o[2], o[3]));
    } else {
        for (int e = 0; e < 4; ++e)
            if (gxi + e < a.nx) dst[e] = o[e];
    }

    if (a.rec.on && k == a.rec.rk) {
        const RecSlot rs = rec_slot(a.rec, gxi, gyi, a.nx);
        if (rs.flags) rec_store(a.rec, rs, n, o);
    }
}

// z pairs of one row from its whole tensor-memory ring v of 2R slots (slot p mod
// 2R holds signed plane p; slot S = vk mod 2R): acc += w_l (q[vk + l] + q[vk - l]),
// l = 1..R ascending, q[vk + R] being the entering qin.
template <int R, int S>
__device__ __forceinline__ void z_pairs_ring(float2 &lo, float2 &hi, const float2 *wz2, const float4 (&v)[2 * R],
                                             const float4 qin)
{
    constexpr int M = 2 * R - 1;   // ring slots - 1
#pragma unroll
    for (int l = 1; l <= R; ++l) {
        const float4 up = l == R ? qin : v[(S + l) & M];
        const float4 dn = v[(S - l + 2 * R) & M];
        lo = __ffma2_rn(wz2[l], __fadd2_rn(make_float2(up.x, up.y), make_float2(dn.x, dn.y)), lo);
        hi = __ffma2_rn(wz2[l], __fadd2_rn(make_float2(up.z, up.w), make_float2(dn.z, dn.w)), hi);
    }
}

// One CTA's work: tile (bx, by), z chunk bz, of the step u^n -> u^{n+1}.
// tm_cur maps u^n with the halo box (ring A), tm_ctile u^n with the tile box
// (the z-queue entries in ring B), tm_prev and tm_kappa the other ring B tiles.
// INJ compiles in the injection lattice (adjoint runs only: the extra branch
// in the store path costs about 6 % when present).  GRAD turns the sweep into
// the adjoint's velocity-gradient term: `cur` is the forward level a = u^n,
// ring B carries z (tm_prev), kappa and the gradient (tm_grad), and each point
// gets grad += a.c2dt z (L a) / sqrt(kappa), written over the gradient (`prev`).
// DEP: the launch is a programmatic dependent of the previous step's: the CTA
// sets up its barriers (and tensor memory) before it waits for that step to
// complete, then takes its time index itself (`n` is ignored).
template <int R, int TX, int TY, int LA, bool INJ, bool GRAD = false, bool DEP = false>
__device__ __forceinline__ void iso_body(const CUtensorMap *tm_cur, const CUtensorMap *tm_prev,
                                         const CUtensorMap *tm_kappa, const CUtensorMap *tm_ctile, const IsoArgs &a,
                                         float *prev, const float *cur, int n, const int bx, const int by,
                                         const int bz, const CUtensorMap *tm_grad = nullptr)
{
    using C = IsoCfg<R, TX, TY, LA, GRAD ? 3 : 2>;
    constexpr bool TQ = C::TQ;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *ringA = reinterpret_cast<float *>(smem_raw);
    float *ringB = reinterpret_cast<float *>(smem_raw + C::OFF_B);
    uint64_t *fullA = reinterpret_cast<uint64_t *>(smem_raw + C::OFF_BAR);
    uint64_t *emptyA = fullA + C::NA;
    uint64_t *fullB = emptyA + C::NA;
    uint64_t *emptyB = fullB + C::NB;
    // [0] n, [1] abort, [2..3] issue counts, [4] step_prologue's, [5] tensor-memory address
    int *sh = reinterpret_cast<int *>(emptyB + C::NB);
    uint32_t *sh_tmem = reinterpret_cast<uint32_t *>(sh + 5);
    volatile int *sh_abort = sh + 1;

    const int tid = threadIdx.x;
    const int x0 = bx * TX, y0 = by * TY;
    const int z0 = a.zb + bz * a.zchunk;             // planes [zb, nz - ztop) of this launch
    const int z1 = min(z0 + a.zchunk, a.nz - a.ztop);
    // At radius 8 the odd chunks sweep downward, so that the two chunks meeting at
    // a boundary prime their z queues from the same 2R planes at the same time
    // (512^3, interleaved in one process: 338.7 vs 327.6 Gpts/s, although DRAM
    // reads rose by 1 %; radius 4 lost 0.9 % and sweeps upward only).  Iteration
    // u works on plane k = k0 + sgn u; the z sums are symmetric pairs
    // (q[k + l] + q[k - l]) whose operands only change places, so the result does
    // not depend on the direction.
    const int sgn = (R >= 8 && (bz & 1)) ? -1 : 1;
    const int k0 = sgn > 0 ? z0 : z1 - 1;
    const int nit = z1 - z0;

    if (tid == 0) {
        for (int s = 0; s < C::NA; ++s) {
            mbar_init(&fullA[s], 1);
            mbar_init(&emptyA[s], C::NCW);
        }
        for (int s = 0; s < C::NB; ++s) {
            mbar_init(&fullB[s], 1);
            mbar_init(&emptyB[s], C::NCW);
        }
        fence_mbar_init();
        sh[0] = n;
        sh[1] = 0;
        sh[2] = 0;
        sh[3] = 0;
    }
    if (tid == C::NC) {
        prefetch_tmap(tm_cur);
        prefetch_tmap(tm_prev);
        prefetch_tmap(tm_kappa);
        prefetch_tmap(tm_ctile);
    }
    if constexpr (TQ) {
        __syncwarp();
        if (tid < 32) tmem_alloc(sh_tmem, C::TMEM_COLS);
    }
    if constexpr (DEP) {
        // Nothing above reads what the previous step writes.  From here on the
        // time index, u^n and the tables (a preceding kernel may have written
        // them) must be that step's.
        griddep_wait();
        if (tid == 0) sh[0] = step_take(a.st, a.ncta, 0x7fffffff, a.hold != 0);
    }
    float *sgz = reinterpret_cast<float *>(smem_raw + C::OFF_GZ);   // z damping factors of the chunk
    for (int i = tid; i < z1 - z0; i += C::NT) sgz[i] = a.gz[z0 + i];
    if constexpr (TQ) tmem_fence_before_sync();
    __syncthreads();
    if constexpr (TQ) tmem_fence_after_sync();
    if constexpr (DEP) n = sh[0];
    bool failed = false;

    if (tid >= C::NC) {
        // ------------------------------------------------------------ producer warp
        if (tid == C::NC) {
            int a_end = 0, b_end = 0;               // iterations issued: A [0, a_end), B [0, b_end)
            bool ok = true;
            // test hook (fd_debug_skip_copy): CTA (0,0,0) withholds one plane's copy,
            // so that its consumers' bounded wait runs out and the launch reports a
            // timeout; every wait on that path is bounded
            const int skip = (bx == 0 && by == 0 && bz == 0) ? a.skip_plane1 - 1 : -1;
            auto issue_a = [&](int u, int p) {
                if (p == skip) {
                    a_end = u + 1;
                    return;
                }
                const int s = u % C::NA;
                if (u >= C::NA && !mbar_wait_bounded(&emptyA[s], ((u / C::NA) - 1) & 1, kWaitLimit)) {
                    ok = false;
                    return;
                }
                mbar_arrive_expect_tx(&fullA[s], C::SLOT_A * 4);
                tma_load_3d(ringA + s * C::SLOT_A, tm_cur, &fullA[s], x0 - R, y0 - R, p);
                a_end = u + 1;
            };
            auto issue_b = [&](int u, int k) {
                const int s = u % C::NB;
                if (u >= C::NB && !mbar_wait_bounded(&emptyB[s], ((u / C::NB) - 1) & 1, kWaitLimit)) {
                    ok = false;
                    return;
                }
                mbar_arrive_expect_tx(&fullB[s], C::SLOT_B * 4);
                float *dst = ringB + s * C::SLOT_B;
                tma_load_3d(dst, tm_prev, &fullB[s], x0, y0, k);
                tma_load_3d(dst + TX * TY, tm_kappa, &fullB[s], x0, y0, k);
                if (GRAD) tma_load_3d(dst + 2 * TX * TY, tm_grad, &fullB[s], x0, y0, k);
                // the z-queue entry: plane k + sgn R (zeros outside the grid)
                tma_load_3d(dst + (C::NBT_ALL - 1) * TX * TY, tm_ctile, &fullB[s], x0, y0, k + sgn * R);
                b_end = u + 1;
            };
            for (int u = 0; ok && u < nit; ++u) {
                if (*sh_abort) break;
                const int k = k0 + sgn * u;
                issue_a(u, k);
                if (ok) issue_b(u, k);
            }
            if (!ok) {
                *sh_abort = 1;
                failed = true;
            }
            sh[2] = a_end;
            sh[3] = b_end;
        }
    } else if constexpr (TQ) {
        // ------------------------------------------------------------ consumer warps (two rows each)
        // Thread (tx, tr) owns 4 consecutive x points of tile rows 2 tr and 2 tr + 1.
        // Their y neighbours overlap, so each staged row above and below is read
        // once for both: 16 float4 reads per 8 points instead of 32.  Per point the
        // arithmetic, and its order, is that of the one-row form.
        const int tx = tid % C::NTX, tr = tid / C::NTX;
        const int lane = tid & 31;
        const int gxi = x0 + 4 * tx, gy0 = y0 + 2 * tr;
        const bool xin = gxi < a.nx;
        const bool act[2] = {xin && gy0 < a.ny, xin && gy0 + 1 < a.ny};
        const long long rowoff0 = (long long)gy0 * a.pitch + gxi;
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const int own = (2 * tr + R) * C::SW + R + 4 * tx;   // row 0's float4 in a ring A slot (row 1: + SW)
        const int ownb = 2 * tr * TX + 4 * tx;               // row 0's float4 in a ring B tile (row 1: + TX)

        // z queues in my tensor-memory lane, indexed by the signed plane index
        // v = sgn p (the sweep then always runs towards larger v): row e's values of
        // v = vk - R .. vk + R - 1 in columns 64 e + [0, 64), v in slot v mod 16 at
        // 4 s.  The plane of vk + R enters from ring B.
        const uint32_t tl = *sh_tmem + ((uint32_t)(32 * (tid / 32)) << 16);
        const int vk0 = sgn * k0;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
#pragma unroll
            for (int m0 = 0; m0 < 2 * R; m0 += 8) {
                float4 v[8];   // eight loads in flight before their stores
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const int p = sgn * (vk0 - R + m0 + m);
                    v[m] = (act[e] && p >= 0 && p < a.nz) ? ld_nc_na(cur + p * a.plane + rowoff0 + e * a.pitch)
                                                          : zero4;
                }
                __syncwarp();
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    tmem_st4(tl + C::QC * e + 4 * (uint32_t)((vk0 - R + m0 + m) & (C::QS - 1)), v[m]);
                }
            }
        }
        float4 g4 = zero4;
        float gyv[2] = {0.f, 0.f};
        if (xin) g4 = *reinterpret_cast<const float4 *>(a.gx + gxi);
#pragma unroll
        for (int e = 0; e < 2; ++e)
            if (act[e]) gyv[e] = a.gy[gy0 + e];

        // tcgen05 loads and stores are warp-collective: every warp takes each
        // branch as a whole, so the abort flag and each bounded wait are agreed
        // across the warp.
        bool ok = true;
        for (int ub = 0; ok && ub < nit; ++ub) {
            const int k = k0 + sgn * ub, vk = sgn * k;
            if (!__all_sync(0xffffffffu, *sh_abort == 0)) {
                ok = false;
                break;
            }
            const int sb = ub % C::NB;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&fullB[sb], (ub / C::NB) & 1, kWaitLimit))) {
                ok = false;
                break;
            }
            const float *tb = ringB + sb * C::SLOT_B;
            float4 qin[2], pv[2], kv[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                qin[e] = *reinterpret_cast<const float4 *>(tb + (C::NBT_ALL - 1) * TX * TY + ownb + e * TX);
                pv[e] = *reinterpret_cast<const float4 *>(tb + ownb + e * TX);
                kv[e] = *reinterpret_cast<const float4 *>(tb + TX * TY + ownb + e * TX);
            }
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&fullA[ub % C::NA], (ub / C::NA) & 1, kWaitLimit))) {
                ok = false;
                break;
            }
            const float gz = sgz[k - z0];
            const int sa = ub % C::NA;
            const float *t = ringA + sa * C::SLOT_A;

            // x windows: floats [4tx - R, 4tx + 4 + R) of both rows of plane k
            float xw[2][4 + 2 * R];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float *rw = t + own + e * C::SW - R;
#pragma unroll
                for (int m = 0; m < (4 + 2 * R) / 4; ++m) {
                    const float4 v = *reinterpret_cast<const float4 *>(rw + 4 * m);
                    xw[e][4 * m + 0] = v.x; xw[e][4 * m + 1] = v.y; xw[e][4 * m + 2] = v.z; xw[e][4 * m + 3] = v.w;
                }
            }
            // centre, then x pairs, per point, on point pairs (0, 1) and (2, 3): for
            // even l both operands are halves of loaded float4s, for odd l the two
            // scalar sums land in a register pair (per lane the rounding of fmaf)
            float2 lo[2], hi[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float *w = xw[e];
                const float2 w02 = make_float2(a.w0, a.w0);
                lo[e] = __fmul2_rn(w02, make_float2(w[R], w[R + 1]));
                hi[e] = __fmul2_rn(w02, make_float2(w[R + 2], w[R + 3]));
#pragma unroll
                for (int l = 1; l <= R; ++l) {
                    float2 slo, shi;
                    if ((l & 1) == 0) {
                        slo = __fadd2_rn(make_float2(w[R + l], w[R + 1 + l]), make_float2(w[R - l], w[R + 1 - l]));
                        shi = __fadd2_rn(make_float2(w[R + 2 + l], w[R + 3 + l]),
                                         make_float2(w[R + 2 - l], w[R + 3 - l]));
                    } else {
                        slo = make_float2(w[R + l] + w[R - l], w[R + 1 + l] + w[R + 1 - l]);
                        shi = make_float2(w[R + 2 + l] + w[R + 2 - l], w[R + 3 + l] + w[R + 3 - l]);
                    }
                    lo[e] = __ffma2_rn(a.wxy2[l], slo, lo[e]);
                    hi[e] = __ffma2_rn(a.wxy2[l], shi, hi[e]);
                }
            }
            auto pair = [&](int e, const float2 w, const float4 &up, const float4 &dn) {
                lo[e] = __ffma2_rn(w, __fadd2_rn(make_float2(up.x, up.y), make_float2(dn.x, dn.y)), lo[e]);
                hi[e] = __ffma2_rn(w, __fadd2_rn(make_float2(up.z, up.w), make_float2(dn.z, dn.w)), hi[e]);
            };
            // y pairs: at l, row 0 takes rows (l, -l) and row 1 rows (l + 1, 1 - l),
            // relative to row 0; rows 0 and 1 themselves are the x windows' centres
            float4 up0 = make_float4(xw[1][R], xw[1][R + 1], xw[1][R + 2], xw[1][R + 3]);
            float4 dn1 = make_float4(xw[0][R], xw[0][R + 1], xw[0][R + 2], xw[0][R + 3]);
#pragma unroll
            for (int l = 1; l <= R; ++l) {
                const float4 dn0 = *reinterpret_cast<const float4 *>(t + own - l * C::SW);
                const float4 up1 = *reinterpret_cast<const float4 *>(t + own + (l + 1) * C::SW);
                pair(0, a.wxy2[l], up0, dn0);
                pair(1, a.wxy2[l], up1, dn1);
                up0 = up1;
                dn1 = dn0;
            }
            // this warp no longer reads plane k from either ring: order its plain
            // reads before the producer's next copies into these slots
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&emptyA[sa]);
                mbar_arrive(&emptyB[sb]);
            }
            // z pairs from the tensor-memory queues
            if constexpr (R == 8 || R == 4) {
                // per row, the whole ring of 2R slots in one load from a fixed
                // address, then pairs l = 1..R at slots (vk + l) and (vk - l) mod 2R,
                // selected through a switch on vk mod 2R (vk + R is the entering one)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    float4 v[2 * R];
                    __syncwarp();
                    if constexpr (R == 8)
                        tmem_ld_ring(tl + C::QC * e, v);
                    else
                        tmem_ld_ring8(tl + C::QC * e, v);
                    switch (vk & (2 * R - 1)) {
#define FD_ZP(S) \
    case S: z_pairs_ring<R, (S) & (2 * R - 1)>(lo[e], hi[e], a.wz2, v, qin[e]); break;
                        FD_ZP(0) FD_ZP(1) FD_ZP(2) FD_ZP(3) FD_ZP(4) FD_ZP(5) FD_ZP(6) FD_ZP(7)
                        FD_ZP(8) FD_ZP(9) FD_ZP(10) FD_ZP(11) FD_ZP(12) FD_ZP(13) FD_ZP(14) FD_ZP(15)
#undef FD_ZP
                    }
                }
                const uint32_t cs = tl + 4 * (uint32_t)((vk + R) & (C::QS - 1));
                tmem_st4_2(cs, qin[0], cs + C::QC, qin[1]);
            } else {
                // per row, pairs l = 1..4 then 5..8: signed indices vk + l and vk - l
                // from their slots (vk + 8 is the entering one; its slot still holds
                // vk - 8)
#pragma unroll
                for (int h = 0; h < R / 4; ++h)
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        uint32_t c[8];
                        float4 v[8];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int l = 4 * h + 1 + i;
                            c[2 * i] = tl + C::QC * e + 4 * (uint32_t)((vk + l) & (C::QS - 1));
                            c[2 * i + 1] = tl + C::QC * e + 4 * (uint32_t)((vk - l) & (C::QS - 1));
                        }
                        __syncwarp();
                        tmem_ld4x8(c, v);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int l = 4 * h + 1 + i;
                            pair(e, a.wz2[l], l == R ? qin[e] : v[2 * i], v[2 * i + 1]);
                        }
                    }
                // vk + 8 takes the slot of vk - 8, no longer needed
                const uint32_t cs = tl + 4 * (uint32_t)((vk + R) & (C::QS - 1));
                tmem_st4_2(cs, qin[0], cs + C::QC, qin[1]);
            }

#pragma unroll
            for (int e = 0; e < 2; ++e) {
                if (!act[e]) continue;
                const float acc[4] = {lo[e].x, lo[e].y, hi[e].x, hi[e].y};
                const float cu[4] = {xw[e][R], xw[e][R + 1], xw[e][R + 2], xw[e][R + 3]};
                update_row<INJ>(a, prev, n, k, gxi, gy0 + e, rowoff0 + e * a.pitch, acc, cu, pv[e], kv[e], g4,
                                gyv[e] * gz);
            }
        }
        if (!ok) {
            *sh_abort = 1;
            failed = true;
        }
    } else {
        // ------------------------------------------------------------ consumer warps (one row each)
        const int tx = tid % C::NTX, ty = tid / C::NTX;
        const int lane = tid & 31;
        const int gxi = x0 + 4 * tx, gyi = y0 + ty;
        const bool act = (gyi < a.ny) && (gxi < a.nx);
        const long long rowoff = (long long)gyi * a.pitch + gxi;
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const int own = (ty + R) * C::SW + R + 4 * tx;   // my float4 in a ring A slot
        const int ownb = ty * TX + 4 * tx;               // my float4 in a ring B tile

        // z queue: q[R + m] = my 4 values of plane k + sgn m, m = -R..R
        float4 q[2 * R + 1];
#pragma unroll
        for (int m = 0; m < 2 * R; ++m) {
            const int p = k0 + sgn * (m - R);
            q[m] = (act && p >= 0 && p < a.nz) ? ld_nc_na(cur + p * a.plane + rowoff) : zero4;
        }
        bool ok = true;
        float4 g4 = zero4;
        float gyv = 0.f;
        if (act) {
            g4 = *reinterpret_cast<const float4 *>(a.gx + gxi);
            gyv = a.gy[gyi];
        }

        for (int ub = 0; ok && ub < nit; ++ub) {
            const int k = k0 + sgn * ub;
            if (*sh_abort) {
                ok = false;
                break;
            }
            const int sb = ub % C::NB;
            if (!mbar_wait_bounded(&fullB[sb], (ub / C::NB) & 1, kWaitLimit)) {
                ok = false;
                break;
            }
            const float *tb = ringB + sb * C::SLOT_B;
            // my values of plane k + sgn R enter the queue
            q[2 * R] = *reinterpret_cast<const float4 *>(tb + (C::NBT_ALL - 1) * TX * TY + ownb);
            // plane k of u^n with its halo, in ring A
            if (!mbar_wait_bounded(&fullA[ub % C::NA], (ub / C::NA) & 1, kWaitLimit)) {
                ok = false;
                break;
            }
            const float4 pv = *reinterpret_cast<const float4 *>(tb + ownb);
            const float4 kv = *reinterpret_cast<const float4 *>(tb + TX * TY + ownb);
            const float4 gv = GRAD ? *reinterpret_cast<const float4 *>(tb + 2 * TX * TY + ownb) : zero4;
            const float gz = sgz[k - z0];

            const int sa = ub % C::NA;
            const float *t = ringA + sa * C::SLOT_A;
            // x window: floats [4tx - R, 4tx + 4 + R) of my row of plane k
            float xw[4 + 2 * R];
            const float *rw = t + own - R;
#pragma unroll
            for (int m = 0; m < (4 + 2 * R) / 4; ++m) {
                const float4 v = *reinterpret_cast<const float4 *>(rw + 4 * m);
                xw[4 * m + 0] = v.x; xw[4 * m + 1] = v.y; xw[4 * m + 2] = v.z; xw[4 * m + 3] = v.w;
            }
            // One accumulator per point, terms in a fixed order (centre, x pairs,
            // y pairs, z pairs).  The y and z sums use packed f32x2 FMA / add on
            // the point pairs (0, 1) and (2, 3): per lane the same rounding as
            // fmaf, with half the instructions.
            float acc[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[e] = a.w0 * xw[R + e];
#pragma unroll
            for (int l = 1; l <= R; ++l)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[e] = fmaf(a.wxy[l], xw[R + e + l] + xw[R + e - l], acc[e]);
            float2 lo = make_float2(acc[0], acc[1]), hi = make_float2(acc[2], acc[3]);
#pragma unroll
            for (int l = 1; l <= R; ++l) {
                const float4 up = *reinterpret_cast<const float4 *>(t + own + l * C::SW);
                const float4 dn = *reinterpret_cast<const float4 *>(t + own - l * C::SW);
                lo = __ffma2_rn(a.wxy2[l], __fadd2_rn(make_float2(up.x, up.y), make_float2(dn.x, dn.y)), lo);
                hi = __ffma2_rn(a.wxy2[l], __fadd2_rn(make_float2(up.z, up.w), make_float2(dn.z, dn.w)), hi);
            }
            // this warp no longer reads plane k from either ring: order its plain
            // reads before the producer's next copies into these slots
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&emptyA[sa]);
                mbar_arrive(&emptyB[sb]);
            }
#pragma unroll
            for (int l = 1; l <= R; ++l) {
                lo = __ffma2_rn(a.wz2[l], __fadd2_rn(make_float2(q[R + l].x, q[R + l].y),
                                                     make_float2(q[R - l].x, q[R - l].y)), lo);
                hi = __ffma2_rn(a.wz2[l], __fadd2_rn(make_float2(q[R + l].z, q[R + l].w),
                                                     make_float2(q[R - l].z, q[R - l].w)), hi);
            }
            acc[0] = lo.x;
            acc[1] = lo.y;
            acc[2] = hi.x;
            acc[3] = hi.y;

            if (GRAD && act) {
                // velocity-gradient term: pv holds z, kv kappa, gv the gradient
                const float zu[4] = {pv.x, pv.y, pv.z, pv.w}, ku[4] = {kv.x, kv.y, kv.z, kv.w};
                float o[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) o[e] += a.c2dt * zu[e] * acc[e] * rsqrtf(ku[e]);
                float *dst = prev + k * a.plane + rowoff;
                if (gxi + 3 < a.nx) {
                    st_cs(dst, make_float4(o[0], o[1], o[2], o[3]));
                } else {
                    for (int e = 0; e < 4; ++e)
                        if (gxi + e < a.nx) dst[e] = o[e];
                }
            } else if (act) {
                const float cu[4] = {xw[R], xw[R + 1], xw[R + 2], xw[R + 3]};
                update_row<INJ>(a, prev, n, k, gxi, gyi, rowoff, acc, cu, pv, kv, g4, gyv * gz);
            }
#pragma unroll
            for (int m = 0; m < 2 * R; ++m) q[m] = q[m + 1];
        }
        if (!ok) {
            *sh_abort = 1;
            failed = true;
        }
    }

    if constexpr (TQ) tmem_fence_before_sync();
    const bool any_failed = __syncthreads_or(failed);
    if constexpr (TQ) {
        tmem_fence_after_sync();
        if (tid < 32) tmem_dealloc(*sh_tmem, C::TMEM_COLS);
    }
    if (any_failed && tid == C::NC) {
        // A bounded wait gave up somewhere: record it, then wait (bounded) for the
        // copies still in flight so that none lands in shared memory after exit.
        atomicOr(&a.st->err, kErrTmaTimeout);
        atomicCAS(&a.st->err_info, 0, 1 + (int)(blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)));
        const int a_end = sh[2], b_end = sh[3];   // iterations issued
        for (int u = max(0, a_end - C::NA); u < a_end; ++u)
            mbar_wait_bounded(&fullA[u % C::NA], (u / C::NA) & 1, kWaitLimit);
        for (int u = max(0, b_end - C::NB); u < b_end; ++u)
            mbar_wait_bounded(&fullB[u % C::NB], (u / C::NB) & 1, kWaitLimit);
    }
}


template <int R, int TX, int TY, int LA, bool INJ>
__global__ void __launch_bounds__(IsoCfg<R, TX, TY, LA>::NT, IsoCfg<R, TX, TY, LA>::MINB)
    iso_sweep_kernel(const __grid_constant__ CUtensorMap tm_cur, const __grid_constant__ CUtensorMap tm_prev,
                     const __grid_constant__ CUtensorMap tm_kappa, const __grid_constant__ CUtensorMap tm_ctile,
                     const __grid_constant__ IsoArgs a)
{
    // the next step's CTAs may start their set-up while this step's last ones run
    griddep_launch_dependents();
    iso_body<R, TX, TY, LA, INJ, false, true>(&tm_cur, &tm_prev, &tm_kappa, &tm_ctile, a, a.prev, a.cur, 0, blockIdx.x,
                                              blockIdx.y, blockIdx.z);
}

// Batched step: one launch advances every member shot of a batch by one step.
// Block b takes work item items[b] = (shot, tile x, tile y, z chunk); the shot's
// time index selects which of its two wavefield buffers holds u^n, so a graph
// of these launches replays without per-step arguments.  Shots that reached
// their last step skip their items.
template <int R, int TX, int TY, int LA>
__global__ void __launch_bounds__(IsoCfg<R, TX, TY, LA>::NT, IsoCfg<R, TX, TY, LA>::MINB)
    iso_batch_kernel(const int4 *__restrict__ items, const BatchShot *__restrict__ shots)
{
    using C = IsoCfg<R, TX, TY, LA>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int4 it = items[blockIdx.x];
    const BatchShot &b = shots[it.x];
    // The shot's parameters are read every plane: keep a copy in shared memory
    // (after the largest z-chunk table) rather than in global memory.
    IsoArgs *sa = reinterpret_cast<IsoArgs *>(smem_raw + C::OFF_GZ + 4 * kMaxChunk);
    static_assert(sizeof(IsoArgs) % 16 == 0, "IsoArgs copies as int4");
    for (int i = threadIdx.x; i < (int)(sizeof(IsoArgs) / 16); i += blockDim.x)
        reinterpret_cast<int4 *>(sa)[i] = reinterpret_cast<const int4 *>(&b.a)[i];
    const int n = step_prologue(b.a.st, b.ncta, b.n_end, reinterpret_cast<int *>(smem_raw + C::OFF_GZ - 16));
    if (n < 0) return;
    const int c = b.cur0 ^ ((n - b.n0) & 1);      // buffer holding u^n
    if (threadIdx.x == C::NC) {
        // the maps sit in the batch's descriptor table, rewritten by host copies
        // whenever the membership changes: the issuing thread acquires them
        fence_tmap_acquire(&b.halo[c]);
        fence_tmap_acquire(&b.tile[0]);
        fence_tmap_acquire(&b.tile[1]);
        fence_tmap_acquire(&b.kappa);
    }
    iso_body<R, TX, TY, LA, false>(&b.halo[c], &b.tile[c ^ 1], &b.kappa, &b.tile[c], *sa, b.buf[c ^ 1], b.buf[c], n, it.y,
                                   it.z, it.w);
}

// ---------------------------------------------------------------------------

constexpr int cmax(int x, int y) { return x > y ? x : y; }

template <int R, int TX, int TY, int LA, bool INJ>
static cudaError_t launch_ti(const IsoMaps &tm, const IsoArgs &a0, cudaStream_t s)
{
    using C = IsoCfg<R, TX, TY, LA>;
    constexpr int smem_max = cmax(C::SMEM + 4 * kMaxChunk, C::SMEM_FLOOR);
    static std::atomic<bool> attr_set[64];   // per device; host threads may launch at once
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev].load(std::memory_order_acquire)) {
        cudaError_t e = cudaFuncSetAttribute(iso_sweep_kernel<R, TX, TY, LA, INJ>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev].store(true, std::memory_order_release);
    }
    IsoArgs a = a0;
    const int zn = a.nz - a.ztop - a.zb;   // planes of this launch
    if (zn <= 0) return cudaErrorInvalidValue;
    dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (zn + a.zchunk - 1) / a.zchunk);
    a.ncta = grid.x * grid.y * grid.z;
    const int smem = cmax(C::SMEM + 4 * ((a.zchunk + 3) / 4 * 4), C::SMEM_FLOOR);
    // Programmatic stream serialisation: consecutive steps overlap one CTA's
    // set-up with the previous step's last CTAs (each CTA waits for that step
    // to complete before it reads anything the step writes).  The tensor-memory
    // form allocates its columns before that wait; shared memory keeps at most
    // three of its CTAs on an SM, of either step, so 3 x 128 of the 512 columns
    // always suffice.  Measured at 512^3: +0.7 % for radius 4, +0.8 % for the
    // radius-8 tensor-memory form.
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(C::NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, iso_sweep_kernel<R, TX, TY, LA, INJ>, tm.cur, tm.prev, tm.kappa, tm.cur_tile, a);
}

template <int R, int TX, int TY, int LA>
static cudaError_t launch_t(const IsoMaps &tm, const IsoArgs &a, cudaStream_t s)
{
    return a.inj.on ? launch_ti<R, TX, TY, LA, true>(tm, a, s) : launch_ti<R, TX, TY, LA, false>(tm, a, s);
}

template <int R, int TX, int TY, int LA>
static cudaError_t launch_b(const int4 *items, int nitems, const BatchShot *shots, int max_zchunk, cudaStream_t s)
{
    using C = IsoCfg<R, TX, TY, LA>;
    constexpr int smem = cmax(C::SMEM + 4 * kMaxChunk + (int)sizeof(IsoArgs), C::SMEM_FLOOR);
    (void)max_zchunk;
    static std::atomic<bool> attr_set[64];   // per device; host threads may launch at once
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev].load(std::memory_order_acquire)) {
        cudaError_t e = cudaFuncSetAttribute(iso_batch_kernel<R, TX, TY, LA>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev].store(true, std::memory_order_release);
    }
    if (nitems <= 0) return cudaSuccess;
    iso_batch_kernel<R, TX, TY, LA><<<nitems, C::NT, smem, s>>>(items, shots);
    return cudaGetLastError();
}

// Velocity-gradient sweep of the adjoint (fd_grad_accumulate): the same
// pipeline over a = u^n, with z, kappa and the gradient in ring B.  It does not
// advance the grid's time index.
template <int R, int TX, int TY, int LA>
__global__ void __launch_bounds__(IsoCfg<R, TX, TY, LA, 3>::NT, IsoCfg<R, TX, TY, LA, 3>::MINB)
    iso_grad_kernel(const __grid_constant__ CUtensorMap tm_a, const __grid_constant__ CUtensorMap tm_z,
                    const __grid_constant__ CUtensorMap tm_kappa, const __grid_constant__ CUtensorMap tm_grad,
                    const __grid_constant__ CUtensorMap tm_atile, const __grid_constant__ IsoArgs a)
{
    iso_body<R, TX, TY, LA, false, true>(&tm_a, &tm_z, &tm_kappa, &tm_atile, a, a.prev, a.cur, 0, blockIdx.x,
                                         blockIdx.y, blockIdx.z, &tm_grad);
}

template <int R, int TX, int TY, int LA>
static cudaError_t launch_g(const IsoMaps &tm, const CUtensorMap &tm_grad, const IsoArgs &a0, cudaStream_t s)
{
    using C = IsoCfg<R, TX, TY, LA, 3>;
    constexpr int smem_max = C::SMEM + 4 * kMaxChunk;
    static std::atomic<bool> attr_set[64];   // per device; host threads may launch at once
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev].load(std::memory_order_acquire)) {
        cudaError_t e = cudaFuncSetAttribute(iso_grad_kernel<R, TX, TY, LA>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev].store(true, std::memory_order_release);
    }
    IsoArgs a = a0;
    dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (a.nz + a.zchunk - 1) / a.zchunk);
    a.ncta = grid.x * grid.y * grid.z;
    const int smem = C::SMEM + 4 * ((a.zchunk + 3) / 4 * 4);
    iso_grad_kernel<R, TX, TY, LA><<<grid, C::NT, smem, s>>>(tm.cur, tm.prev, tm.kappa, tm_grad, tm.cur_tile, a);
    return cudaGetLastError();
}

Launch iso_grad_launch(int R, int nx, int ny, int nz)
{
    // the gradient sweep keeps the register queue: radius 4 in 64 x 16 tiles (two
    // CTAs per SM), radius 8 in 32 x 16 (three)
    Launch L;
    L.tx = R == 8 ? 32 : 64;
    L.ty = 16;
    L.lookahead = R == 8 ? 2 : 3;
    L.zchunk = R == 8 ? default_zchunk(L, nx, ny, nz, 4096)
                      : wave_zchunk(L, nx, ny, nz, (long)device_sm_count() * IsoCfg<4, 64, 16, 3>::MINB, 2 * R);
    return L;
}

cudaError_t launch_iso_grad(int R, const Launch &L, const IsoMaps &tm, const CUtensorMap &tm_grad, const IsoArgs &a,
                            cudaStream_t s)
{
    if (R == 4 && L.tx == 64 && L.ty == 16 && L.lookahead == 3) return launch_g<4, 64, 16, 3>(tm, tm_grad, a, s);
    if (R == 8 && L.tx == 32 && L.ty == 16 && L.lookahead == 2) return launch_g<8, 32, 16, 2>(tm, tm_grad, a, s);
    return cudaErrorInvalidConfiguration;
}

// The (R, tile, lookahead) combinations built into the library.
#define FD_ISO_CONFIGS(X) \
    X(4, 64, 16, 3)       \
    X(4, 64, 16, 4)       \
    X(4, 64, 16, 2)       \
    X(4, 64, 8, 3)        \
    X(4, 128, 8, 3)       \
    X(4, 32, 16, 3)       \
    X(4, 32, 32, 2)       \
    X(4, 32, 32, 3)       \
    X(8, 64, 8, 2)        \
    X(8, 64, 8, 3)        \
    X(8, 32, 16, 2)       \
    X(8, 32, 32, 2)

cudaError_t launch_iso(int R, const Launch &L, const IsoMaps &tm, const IsoArgs &a, cudaStream_t s)
{
#define FD_ISO_CASE(R_, TX_, TY_, LA_) \
    if (R == R_ && L.tx == TX_ && L.ty == TY_ && L.lookahead == LA_) return launch_t<R_, TX_, TY_, LA_>(tm, a, s);
    FD_ISO_CONFIGS(FD_ISO_CASE)
#undef FD_ISO_CASE
    return cudaErrorInvalidConfiguration;
}

cudaError_t launch_iso_batch(int R, const Launch &L, const int4 *items, int nitems, const BatchShot *shots,
                             int max_zchunk, cudaStream_t s)
{
#define FD_ISO_BCASE(R_, TX_, TY_, LA_)                                \
    if (R == R_ && L.tx == TX_ && L.ty == TY_ && L.lookahead == LA_) \
        return launch_b<R_, TX_, TY_, LA_>(items, nitems, shots, max_zchunk, s);
    FD_ISO_CONFIGS(FD_ISO_BCASE)
#undef FD_ISO_BCASE
    return cudaErrorInvalidConfiguration;
}

bool iso_config_built(int R, const Launch &L)
{
#define FD_ISO_BUILT(R_, TX_, TY_, LA_) \
    if (R == R_ && L.tx == TX_ && L.ty == TY_ && L.lookahead == LA_) return true;
    FD_ISO_CONFIGS(FD_ISO_BUILT)
#undef FD_ISO_BUILT
    return false;
}

Launch iso_default_launch(int R, int nx, int ny, int nz)
{
    Launch L;
    if (R == 4) {
        // three CTAs of 32 x 32 per SM, z queues in tensor memory, two rows per
        // thread (512^3: 401.7 vs 394.6 Gpts/s for the one-row 64 x 16 form,
        // interleaved in one process)
        L.tx = 32;
        L.ty = 32;
        L.lookahead = 3;
        L.zchunk = wave_zchunk(L, nx, ny, nz, (long)device_sm_count() * IsoCfg<4, 32, 32, 3>::MINB, 2 * R);
    } else {
        // two CTAs of 32 x 32 per SM (z queues in tensor memory, two rows per thread)
        L.tx = 32;
        L.ty = 32;
        L.lookahead = 2;
        L.zchunk = wave_zchunk(L, nx, ny, nz, (long)device_sm_count() * IsoCfg<8, 32, 32, 2>::MINB, 2 * R);
    }
    return L;
}

bool iso_supported(int R) { return R == 4 || R == 8; }

}  // namespace fdk
