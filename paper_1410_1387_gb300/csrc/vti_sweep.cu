// VTI sweep: one leapfrog step (Eq. 3) of the pseudo-acoustic system of
// Eqs. 1-2 with the symmetric x-y stencil of radius R_xy (Eq. 4) and the
// per-plane z stencil of radius R_z (Eq. 5), damping layer, source and
// receiver lattice fused in:
//   Hp = (d_xx + d_yy) p,  Dq = d_zz q (weights of plane k, dz absorbed)
//   p^{n+1} = G (2p - G p_prev + kx Hp + kz Dq + s)
//   q^{n+1} = G (2q - G q_prev + kn Hp + kz Dq [+ s])
// p needs only x-y neighbours and q only z neighbours (Sec. 1).  Warp-specialised
// TMA pipeline, as the isotropic sweep:
//   * ring A: plane k of p^n with an R_xy halo (zero fill outside the grid is
//     the zero halo), used once, as the centre plane;
//   * ring B: the TX x TY tiles of p_prev, q_prev, kx, kn, kz of plane k and of
//     q^n of plane k + R_z (the value that enters the z queue at step k);
//   * each consumer thread keeps the 2 R_z + 1 z neighbours of its 4 q values in
//     registers; the new levels overwrite the older ones in place.  At R_z = 8 in
//     32 x 32 tiles (the default) the queues live in tensor memory instead and
//     each thread takes two adjacent rows, which share their y-neighbour reads of
//     p (the smaller tile also cuts ring A's halo from 5.5x to 3.1x the tile).
// Compulsory HBM traffic: 36 bytes per point update (read p, q, p_prev, q_prev,
// kx, kn, kz; write p, q).
#include <atomic>

#include "fd_internal.h"
#include "launch_shape.h"
#include "ptx.cuh"
#include "rec_slot.cuh"
#include "tmem.cuh"

namespace fdk {

constexpr long long kVtiWaitLimit = 2000000000LL;   // ~1 s

template <int RXY, int RZ, int TX, int TY, int LA>
struct VtiCfg {
    static constexpr int NTX = TX / 4;
    // R_z = 8 in 32 x 32 tiles keeps q's z queues in tensor memory, which frees the
    // registers for two tile rows per thread: the rows share their y-neighbour
    // reads of p (24 float4 per 8 points instead of 48 at R_xy = 12).
    static constexpr bool TQ = (RZ == 8 && TX == 32 && TY == 32);
    static constexpr int RPT = TQ ? 2 : 1;          // tile rows per consumer thread
    static constexpr int NC = NTX * TY / RPT;
    static constexpr int TMEM_COLS = 128;           // two rows x 16 slots x 4 columns
    static constexpr int NCW = NC / 32;
    static constexpr int NT = NC + 32;
    static constexpr int SW = TX + 2 * RXY;
    static constexpr int SH = TY + 2 * RXY;
    static constexpr int SLOT_A = SW * SH;
    static constexpr int TILE = TX * TY;
    static constexpr int ZROW = vti_zrow(RZ);       // paired z weights and G_z of the plane
    // p_prev, q_prev, kx, kn, kz, q ahead, then the z row (slots stay 128-byte aligned)
    static constexpr int SLOT_B = 6 * TILE + (ZROW + 31) / 32 * 32;
    static constexpr int NA = LA + 1;
    static constexpr int NB = LA + 1;
    static constexpr int OFF_B = NA * SLOT_A * 4;
    static constexpr int OFF_BAR = OFF_B + NB * SLOT_B * 4;
    static constexpr int SMEM = OFF_BAR + 8 * (2 * NA + 2 * NB) + 32;   // barriers, then 8 ints
    static constexpr int NW = 2 * RZ + 1;
    static_assert(TX % 4 == 0 && RXY % 4 == 0, "x alignment");
    static_assert(NC % 32 == 0, "whole consumer warps");
    static_assert((SLOT_A * 4) % 128 == 0 && (TILE * 4) % 128 == 0, "slot alignment");
    static_assert(SW <= 256 && SH <= 256, "TMA box limit");
    static_assert(!TQ || NC == 128, "tensor-memory queues: one consumer warp per lane quarter");
};

// Dq of one row from its tensor-memory ring v (plane p of q in slot p mod 16,
// planes k - 8 .. k + 7) when k mod 16 = S, and the entering plane q8 = q^{k+8}:
// sum over m = 0..16 of w2[m] q^{k-8+m}, in ascending m as the register form
// does, on the point pairs (0, 1) and (2, 3); qc receives q^k.
template <int S>
__device__ __forceinline__ void vti_dq_slots(const float4 (&v)[16], const float4 q8, const float2 (&w2)[17],
                                             float2 &lo, float2 &hi, float4 &qc)
{
    lo = make_float2(0.f, 0.f);
    hi = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < 17; ++m) {
        const float4 u = m == 16 ? q8 : v[(S + 8 + m) & 15];   // plane k - 8 + m
        lo = __ffma2_rn(w2[m], make_float2(u.x, u.y), lo);
        hi = __ffma2_rn(w2[m], make_float2(u.z, u.w), hi);
    }
    qc = v[S];
}

// The two updates of one thread's 4 points of plane k in row gyi (Eqs. 1-2 in
// the leapfrog of Eq. 3, damping in its deferred form, G = gx * gy * gz), with the
// source and the receivers; the new levels are written over the older ones.
__device__ __forceinline__ void vti_update_row(const VtiArgs &a, const int n, const int k, const int gxi,
                                               const int gyi, const long long rowoff, const float (&hp)[4],
                                               const float (&dq)[4], const float (&pcu)[4], const float (&qc)[4],
                                               const float (&ppu)[4], const float (&qpu)[4], const float (&kxu)[4],
                                               const float (&knu)[4], const float (&kzu)[4], const float (&gu)[4],
                                               const float gyz)
{
    float op[4], oq[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float G = gu[e] * gyz;
        const float zt = kzu[e] * dq[e];
        op[e] = fmaf(kxu[e], hp[e], fmaf(2.f, pcu[e], -G * ppu[e])) + zt;
        oq[e] = fmaf(knu[e], hp[e], fmaf(2.f, qc[e], -G * qpu[e])) + zt;
    }
    if (k == a.src.sz && gyi == a.src.sy && a.src.sx >= gxi && a.src.sx < gxi + 4 && n < a.src.len) {
        // constant indices only: an index computed at run time would put op and
        // oq in local memory, stored on every update
        const float sv = a.src.tab[n];
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (a.src.sx == gxi + e) {
                op[e] += sv;
                if (a.src.into_q) oq[e] += sv;
            }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float G = gu[e] * gyz;
        op[e] *= G;
        oq[e] *= G;
    }
    float *dp = a.pprev + k * a.plane + rowoff;
    float *dq_ = a.qprev + k * a.plane + rowoff;
    if (gxi + 3 < a.nx) {
        st_cs(dp, make_float4(op[0], op[1], op[2], op[3]));
        st_cs(dq_, make_float4(oq[0], oq[1], oq[2], oq[3]));
    } else {
        for (int e = 0; e < 4; ++e)
            if (gxi + e < a.nx) {
                dp[e] = op[e];
                dq_[e] = oq[e];
            }
    }
    if (a.rec.on && k == a.rec.rk) {
        const RecSlot rs = rec_slot(a.rec, gxi, gyi, a.nx);
        if (rs.flags) rec_store(a.rec, rs, n, op);
    }
}

template <int RXY, int RZ, int TX, int TY, int LA>
__global__ void __launch_bounds__(VtiCfg<RXY, RZ, TX, TY, LA>::NT, 2)
    vti_sweep_kernel(const __grid_constant__ CUtensorMap tm_p, const __grid_constant__ CUtensorMap tm_q,
                     const __grid_constant__ CUtensorMap tm_pp, const __grid_constant__ CUtensorMap tm_qp,
                     const __grid_constant__ CUtensorMap tm_kx, const __grid_constant__ CUtensorMap tm_kn,
                     const __grid_constant__ CUtensorMap tm_kz, const VtiArgs a)
{
    using C = VtiCfg<RXY, RZ, TX, TY, LA>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *ringA = reinterpret_cast<float *>(smem_raw);
    float *ringB = reinterpret_cast<float *>(smem_raw + C::OFF_B);
    uint64_t *fullA = reinterpret_cast<uint64_t *>(smem_raw + C::OFF_BAR);
    uint64_t *emptyA = fullA + C::NA;
    uint64_t *fullB = emptyA + C::NA;
    uint64_t *emptyB = fullB + C::NB;
    // [0] n, [1] abort, [2..3] issue counts, [4] tensor-memory address
    int *sh = reinterpret_cast<int *>(emptyB + C::NB);
    uint32_t *sh_tmem = reinterpret_cast<uint32_t *>(sh + 4);
    volatile int *sh_abort = sh + 1;

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = a.zb + blockIdx.z * a.zchunk;     // planes [zb, nz - ztop) of this launch
    const int z1 = min(z0 + a.zchunk, a.nz - a.ztop);

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
        const int n = *reinterpret_cast<volatile int *>(&a.st->step);
        // the last CTA advances the time index, unless a later part of the step will
        __threadfence();
        if (!a.hold && atomicAdd(&a.st->done, 1u) == a.ncta - 1) {
            a.st->done = 0;
            *reinterpret_cast<volatile int *>(&a.st->step) = n + 1;
            __threadfence();
        }
        sh[0] = n;
        sh[1] = 0;
        sh[2] = z0;
        sh[3] = z0;
    }
    if constexpr (C::TQ) {
        __syncwarp();
        if (tid < 32) tmem_alloc(sh_tmem, C::TMEM_COLS);
        tmem_fence_before_sync();
    }
    __syncthreads();
    if constexpr (C::TQ) tmem_fence_after_sync();
    const int n = sh[0];
    bool failed = false;

    if (tid >= C::NC) {
        // ------------------------------------------------------------ producer warp
        if (tid == C::NC) {
            const CUtensorMap *maps[7] = {&tm_p, &tm_q, &tm_pp, &tm_qp, &tm_kx, &tm_kn, &tm_kz};
            for (const CUtensorMap *m : maps) prefetch_tmap(m);
            int a_end = z0, b_end = z0;
            bool ok = true;
            // test hook (fd_debug_skip_copy): CTA (0,0,0) withholds one plane's copy of
            // p^n, so that its consumers' bounded wait runs out; every wait on that path
            // is bounded
            const int skip = (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) ? a.skip_plane1 - 1 : -1;
            for (int k = z0; ok && k < z1; ++k) {
                if (*sh_abort) break;
                const int u = k - z0;
                const int sa = u % C::NA, sb = u % C::NB;
                if (k != skip) {
                    if (u >= C::NA && !mbar_wait_bounded(&emptyA[sa], ((u / C::NA) - 1) & 1, kVtiWaitLimit)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&fullA[sa], C::SLOT_A * 4);
                    tma_load_3d(ringA + sa * C::SLOT_A, &tm_p, &fullA[sa], x0 - RXY, y0 - RXY, k);
                }
                a_end = k + 1;
                if (u >= C::NB && !mbar_wait_bounded(&emptyB[sb], ((u / C::NB) - 1) & 1, kVtiWaitLimit)) {
                    ok = false;
                    break;
                }
                const bool ahead = k + RZ < a.nz;
                mbar_arrive_expect_tx(&fullB[sb], (ahead ? 6 : 5) * C::TILE * 4 + C::ZROW * 4);
                float *dst = ringB + sb * C::SLOT_B;
                bulk_load(dst + 6 * C::TILE, a.ztab + (long long)k * C::ZROW, C::ZROW * 4, &fullB[sb]);
                tma_load_3d(dst + 0 * C::TILE, &tm_pp, &fullB[sb], x0, y0, k);
                tma_load_3d(dst + 1 * C::TILE, &tm_qp, &fullB[sb], x0, y0, k);
                tma_load_3d(dst + 2 * C::TILE, &tm_kx, &fullB[sb], x0, y0, k);
                tma_load_3d(dst + 3 * C::TILE, &tm_kn, &fullB[sb], x0, y0, k);
                tma_load_3d(dst + 4 * C::TILE, &tm_kz, &fullB[sb], x0, y0, k);
                if (ahead) tma_load_3d(dst + 5 * C::TILE, &tm_q, &fullB[sb], x0, y0, k + RZ);
                b_end = k + 1;
            }
            if (!ok) {
                *sh_abort = 1;
                failed = true;
            }
            sh[2] = a_end;
            sh[3] = b_end;
        }
    } else if constexpr (C::TQ) {
        // ------------------------------------------------------------ consumer warps (two rows each)
        // Thread (tx, tr) owns 4 consecutive x points of tile rows 2 tr and 2 tr + 1;
        // the rows' y neighbours overlap, so each staged row of p above and below is
        // read once for both.  Per point the arithmetic, and its order, is that of
        // the one-row form.  q's z queues live in tensor memory: row e's planes
        // k - RZ .. k + RZ - 1 in columns 64 e + [0, 64), plane p in slot p mod 16.
        const int tx = tid % C::NTX, tr = tid / C::NTX;
        const int gxi = x0 + 4 * tx, gy0 = y0 + 2 * tr;
        const bool xin = gxi < a.nx;
        const bool act[2] = {xin && gy0 < a.ny, xin && gy0 + 1 < a.ny};
        const long long rowoff0 = (long long)gy0 * a.pitch + gxi;
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const int own = (2 * tr + RXY) * C::SW + RXY + 4 * tx;   // row 0's float4 in ring A (row 1: + SW)
        const int ownb = 2 * tr * TX + 4 * tx;                   // row 0's float4 in a ring B tile (row 1: + TX)
        const int lane = tid & 31;
        const uint32_t tl = *sh_tmem + ((uint32_t)(32 * (tid / 32)) << 16);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
#pragma unroll
            for (int m0 = 0; m0 < 2 * RZ; m0 += 8) {
                float4 v[8];   // eight loads in flight before their stores
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const int p = z0 - RZ + m0 + m;
                    v[m] = (act[e] && p >= 0 && p < a.nz) ? ld_nc_na(a.q + p * a.plane + rowoff0 + e * a.pitch)
                                                          : zero4;
                }
                __syncwarp();
#pragma unroll
                for (int m = 0; m < 8; ++m) tmem_st4(tl + 64 * e + 4 * (uint32_t)((z0 - RZ + m0 + m) & 15), v[m]);
            }
        }
        float4 g4 = zero4;
        float gyv[2] = {0.f, 0.f};
        if (xin) g4 = *reinterpret_cast<const float4 *>(a.gx + gxi);
#pragma unroll
        for (int e = 0; e < 2; ++e)
            if (act[e]) gyv[e] = a.gy[gy0 + e];

        // tcgen05 loads and stores are warp-collective: the abort flag and each
        // bounded wait's outcome are agreed across the warp before any branch
        bool ok = true;
        for (int k = z0; ok && k < z1; ++k) {
            if (!__all_sync(0xffffffffu, *sh_abort == 0)) {
                ok = false;
                break;
            }
            const int u = k - z0;
            const int sa = u % C::NA, sb = u % C::NB;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&fullB[sb], (u / C::NB) & 1, kVtiWaitLimit))) {
                ok = false;
                break;
            }
            const float *tb = ringB + sb * C::SLOT_B;
            float4 qin[2];
#pragma unroll
            for (int e = 0; e < 2; ++e)
                qin[e] = (k + RZ < a.nz) ? *reinterpret_cast<const float4 *>(tb + 5 * C::TILE + ownb + e * TX) : zero4;
            const float *zrow = tb + 6 * C::TILE;
            float2 w2[2 * RZ + 1];
#pragma unroll
            for (int m = 0; m < C::NW; ++m) w2[m] = *reinterpret_cast<const float2 *>(zrow + 2 * m);
            const float gz = zrow[2 * C::NW];

            // Dq and the centre q of both rows from the tensor-memory rings
            float2 dq_lo[2], dq_hi[2];
            float4 qc[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                float4 v[16];
                __syncwarp();
                tmem_ld_ring(tl + 64 * e, v);
                switch (k & 15) {
#define FD_VTI_DQ(S_) \
    case S_: vti_dq_slots<S_>(v, qin[e], w2, dq_lo[e], dq_hi[e], qc[e]); break;
                    FD_VTI_DQ(0) FD_VTI_DQ(1) FD_VTI_DQ(2) FD_VTI_DQ(3) FD_VTI_DQ(4) FD_VTI_DQ(5) FD_VTI_DQ(6)
                    FD_VTI_DQ(7) FD_VTI_DQ(8) FD_VTI_DQ(9) FD_VTI_DQ(10) FD_VTI_DQ(11) FD_VTI_DQ(12) FD_VTI_DQ(13)
                    FD_VTI_DQ(14) FD_VTI_DQ(15)
#undef FD_VTI_DQ
                }
            }

            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&fullA[sa], (u / C::NA) & 1, kVtiWaitLimit))) {
                ok = false;
                break;
            }
            const float *t = ringA + sa * C::SLOT_A;
            // Hp: centre, then x pairs (scalar sums, f32x2 FMAs: per lane the
            // rounding of fmaf), then y pairs
            float xw[2][4 + 2 * RXY];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float *rw = t + own + e * C::SW - RXY;
#pragma unroll
                for (int m = 0; m < (4 + 2 * RXY) / 4; ++m) {
                    const float4 v = *reinterpret_cast<const float4 *>(rw + 4 * m);
                    xw[e][4 * m + 0] = v.x; xw[e][4 * m + 1] = v.y; xw[e][4 * m + 2] = v.z; xw[e][4 * m + 3] = v.w;
                }
            }
            float2 lo[2], hi[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float *w = xw[e];
                const float2 w02 = make_float2(a.w0, a.w0);
                lo[e] = __fmul2_rn(w02, make_float2(w[RXY], w[RXY + 1]));
                hi[e] = __fmul2_rn(w02, make_float2(w[RXY + 2], w[RXY + 3]));
#pragma unroll
                for (int l = 1; l <= RXY; ++l) {
                    float2 slo, shi;
                    if ((l & 1) == 0) {
                        slo = __fadd2_rn(make_float2(w[RXY + l], w[RXY + 1 + l]), make_float2(w[RXY - l], w[RXY + 1 - l]));
                        shi = __fadd2_rn(make_float2(w[RXY + 2 + l], w[RXY + 3 + l]),
                                         make_float2(w[RXY + 2 - l], w[RXY + 3 - l]));
                    } else {
                        slo = make_float2(w[RXY + l] + w[RXY - l], w[RXY + 1 + l] + w[RXY + 1 - l]);
                        shi = make_float2(w[RXY + 2 + l] + w[RXY + 2 - l], w[RXY + 3 + l] + w[RXY + 3 - l]);
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
            const float4 pc[2] = {make_float4(xw[0][RXY], xw[0][RXY + 1], xw[0][RXY + 2], xw[0][RXY + 3]),
                                  make_float4(xw[1][RXY], xw[1][RXY + 1], xw[1][RXY + 2], xw[1][RXY + 3])};
            float4 up0 = pc[1], dn1 = pc[0];
#pragma unroll
            for (int l = 1; l <= RXY; ++l) {
                const float4 dn0 = *reinterpret_cast<const float4 *>(t + own - l * C::SW);
                const float4 up1 = *reinterpret_cast<const float4 *>(t + own + (l + 1) * C::SW);
                pair(0, a.wxy2[l], up0, dn0);
                pair(1, a.wxy2[l], up1, dn1);
                up0 = up1;
                dn1 = dn0;
            }
            float4 ppv[2], qpv[2], kxv[2], knv[2], kzv[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float *b = tb + ownb + e * TX;
                ppv[e] = *reinterpret_cast<const float4 *>(b + 0 * C::TILE);
                qpv[e] = *reinterpret_cast<const float4 *>(b + 1 * C::TILE);
                kxv[e] = *reinterpret_cast<const float4 *>(b + 2 * C::TILE);
                knv[e] = *reinterpret_cast<const float4 *>(b + 3 * C::TILE);
                kzv[e] = *reinterpret_cast<const float4 *>(b + 4 * C::TILE);
            }
            // this warp no longer reads plane k from either ring: order its plain
            // reads before the producer's next copies into these slots
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&emptyA[sa]);
                mbar_arrive(&emptyB[sb]);
            }
            // plane k + RZ takes the slot of plane k - RZ, no longer needed
            {
                const uint32_t cs = tl + 4 * (uint32_t)((k + RZ) & 15);
                tmem_st4_2(cs, qin[0], cs + 64, qin[1]);
            }

#pragma unroll
            for (int e = 0; e < 2; ++e) {
                if (!act[e]) continue;
                const int gyi = gy0 + e;
                const float gyz = gyv[e] * gz;
                const float hp[4] = {lo[e].x, lo[e].y, hi[e].x, hi[e].y};
                const float dq[4] = {dq_lo[e].x, dq_lo[e].y, dq_hi[e].x, dq_hi[e].y};
                const float pcu[4] = {pc[e].x, pc[e].y, pc[e].z, pc[e].w};
                const float qcu[4] = {qc[e].x, qc[e].y, qc[e].z, qc[e].w};
                const float ppu[4] = {ppv[e].x, ppv[e].y, ppv[e].z, ppv[e].w};
                const float qpu[4] = {qpv[e].x, qpv[e].y, qpv[e].z, qpv[e].w};
                const float kxu[4] = {kxv[e].x, kxv[e].y, kxv[e].z, kxv[e].w};
                const float knu[4] = {knv[e].x, knv[e].y, knv[e].z, knv[e].w};
                const float kzu[4] = {kzv[e].x, kzv[e].y, kzv[e].z, kzv[e].w};
                const float gu[4] = {g4.x, g4.y, g4.z, g4.w};
                vti_update_row(a, n, k, gxi, gyi, rowoff0 + e * a.pitch, hp, dq, pcu, qcu, ppu, qpu, kxu, knu, kzu,
                               gu, gyz);
            }
        }
        if (!ok) {
            *sh_abort = 1;
            failed = true;
        }
    } else {
        // ------------------------------------------------------------ consumer warps
        const int tx = tid % C::NTX, ty = tid / C::NTX;
        const int lane = tid & 31;
        const int gxi = x0 + 4 * tx, gyi = y0 + ty;
        const bool act = (gyi < a.ny) && (gxi < a.nx);
        const long long rowoff = (long long)gyi * a.pitch + gxi;
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const int own = (ty + RXY) * C::SW + RXY + 4 * tx;
        const int ownb = ty * TX + 4 * tx;

        // q queue: qq[RZ + m] = my 4 q values of plane k + m
        float4 qq[2 * RZ + 1];
#pragma unroll
        for (int m = 0; m < 2 * RZ; ++m) {
            const int p = z0 - RZ + m;
            qq[m] = (act && p >= 0 && p < a.nz) ? ld_nc_na(a.q + p * a.plane + rowoff) : zero4;
        }
        float4 g4 = zero4;
        float gyv = 0.f;
        if (act) {
            g4 = *reinterpret_cast<const float4 *>(a.gx + gxi);
            gyv = a.gy[gyi];
        }
        bool ok = true;
        for (int k = z0; k < z1; ++k) {
            if (*sh_abort) {
                ok = false;
                break;
            }
            const int u = k - z0;
            const int sa = u % C::NA, sb = u % C::NB;
            if (!mbar_wait_bounded(&fullB[sb], (u / C::NB) & 1, kVtiWaitLimit)) {
                ok = false;
                break;
            }
            const float *tb = ringB + sb * C::SLOT_B + ownb;
            const float4 ppv = *reinterpret_cast<const float4 *>(tb + 0 * C::TILE);
            const float4 qpv = *reinterpret_cast<const float4 *>(tb + 1 * C::TILE);
            const float4 kxv = *reinterpret_cast<const float4 *>(tb + 2 * C::TILE);
            const float4 knv = *reinterpret_cast<const float4 *>(tb + 3 * C::TILE);
            const float4 kzv = *reinterpret_cast<const float4 *>(tb + 4 * C::TILE);
            qq[2 * RZ] = (k + RZ < a.nz) ? *reinterpret_cast<const float4 *>(tb + 5 * C::TILE) : zero4;

            // Dq from the plane's z row (weights paired for f32x2), l = -RZ..RZ ascending
            const float *zrow = ringB + sb * C::SLOT_B + 6 * C::TILE;
            float2 dq_lo = make_float2(0.f, 0.f), dq_hi = make_float2(0.f, 0.f);
#pragma unroll
            for (int m = 0; m < C::NW; ++m) {
                const float2 w2 = *reinterpret_cast<const float2 *>(zrow + 2 * m);
                dq_lo = __ffma2_rn(w2, make_float2(qq[m].x, qq[m].y), dq_lo);
                dq_hi = __ffma2_rn(w2, make_float2(qq[m].z, qq[m].w), dq_hi);
            }
            const float gz = zrow[2 * C::NW];

            if (!mbar_wait_bounded(&fullA[sa], (u / C::NA) & 1, kVtiWaitLimit)) {
                ok = false;
                break;
            }
            const float *t = ringA + sa * C::SLOT_A;
            float hp[4];
            {
                // x window [4tx - RXY, 4tx + 4 + RXY), streamed a float4 at a time
                const float *rw = t + own - RXY;
                float xw[4 + 2 * RXY];
#pragma unroll
                for (int m = 0; m < (4 + 2 * RXY) / 4; ++m) {
                    const float4 v = *reinterpret_cast<const float4 *>(rw + 4 * m);
                    xw[4 * m + 0] = v.x; xw[4 * m + 1] = v.y; xw[4 * m + 2] = v.z; xw[4 * m + 3] = v.w;
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) hp[e] = a.w0 * xw[RXY + e];
#pragma unroll
                for (int l = 1; l <= RXY; ++l)
#pragma unroll
                    for (int e = 0; e < 4; ++e) hp[e] = fmaf(a.wxy[l], xw[RXY + e + l] + xw[RXY + e - l], hp[e]);
            }
            const float4 pc = *reinterpret_cast<const float4 *>(t + own);
            // y pairs with packed f32x2 on points (0, 1) and (2, 3)
            float2 hp_lo = make_float2(hp[0], hp[1]), hp_hi = make_float2(hp[2], hp[3]);
#pragma unroll
            for (int l = 1; l <= RXY; ++l) {
                const float4 up = *reinterpret_cast<const float4 *>(t + own + l * C::SW);
                const float4 dn = *reinterpret_cast<const float4 *>(t + own - l * C::SW);
                hp_lo = __ffma2_rn(a.wxy2[l], __fadd2_rn(make_float2(up.x, up.y), make_float2(dn.x, dn.y)), hp_lo);
                hp_hi = __ffma2_rn(a.wxy2[l], __fadd2_rn(make_float2(up.z, up.w), make_float2(dn.z, dn.w)), hp_hi);
            }
            hp[0] = hp_lo.x;
            hp[1] = hp_lo.y;
            hp[2] = hp_hi.x;
            hp[3] = hp_hi.y;
            // this warp no longer reads plane k from either ring: order its plain
            // reads before the producer's next copies into these slots
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&emptyA[sa]);
                mbar_arrive(&emptyB[sb]);
            }
            const float dq[4] = {dq_lo.x, dq_lo.y, dq_hi.x, dq_hi.y};

            if (act) {
                const float pcu[4] = {pc.x, pc.y, pc.z, pc.w};
                const float qc[4] = {qq[RZ].x, qq[RZ].y, qq[RZ].z, qq[RZ].w};
                const float ppu[4] = {ppv.x, ppv.y, ppv.z, ppv.w};
                const float qpu[4] = {qpv.x, qpv.y, qpv.z, qpv.w};
                const float kxu[4] = {kxv.x, kxv.y, kxv.z, kxv.w};
                const float knu[4] = {knv.x, knv.y, knv.z, knv.w};
                const float kzu[4] = {kzv.x, kzv.y, kzv.z, kzv.w};
                const float gu[4] = {g4.x, g4.y, g4.z, g4.w};
                vti_update_row(a, n, k, gxi, gyi, rowoff, hp, dq, pcu, qc, ppu, qpu, kxu, knu, kzu, gu, gyv * gz);
            }
#pragma unroll
            for (int m = 0; m < 2 * RZ; ++m) qq[m] = qq[m + 1];
        }
        if (!ok) {
            *sh_abort = 1;
            failed = true;
        }
    }

    if constexpr (C::TQ) tmem_fence_before_sync();
    const bool any_failed = __syncthreads_or(failed);
    if constexpr (C::TQ) {
        tmem_fence_after_sync();
        if (tid < 32) tmem_dealloc(*sh_tmem, C::TMEM_COLS);
    }
    if (any_failed && tid == C::NC) {
        atomicOr(&a.st->err, kErrTmaTimeout);
        atomicCAS(&a.st->err_info, 0, 1 + (int)(blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)));
        const int a_end = sh[2], b_end = sh[3];
        for (int p = max(z0, a_end - C::NA); p < a_end; ++p) {
            const int u = p - z0;
            mbar_wait_bounded(&fullA[u % C::NA], (u / C::NA) & 1, kVtiWaitLimit);
        }
        for (int p = max(z0, b_end - C::NB); p < b_end; ++p) {
            const int u = p - z0;
            mbar_wait_bounded(&fullB[u % C::NB], (u / C::NB) & 1, kVtiWaitLimit);
        }
    }
}

template <int RXY, int RZ, int TX, int TY, int LA>
static cudaError_t launch_vt(const VtiMaps &tm, const VtiArgs &a0, cudaStream_t s)
{
    using C = VtiCfg<RXY, RZ, TX, TY, LA>;
    static std::atomic<bool> attr_set[64];   // per device; host threads may launch at once
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev].load(std::memory_order_acquire)) {
        cudaError_t e = cudaFuncSetAttribute(vti_sweep_kernel<RXY, RZ, TX, TY, LA>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev].store(true, std::memory_order_release);
    }
    VtiArgs a = a0;
    const int zn = a.nz - a.ztop - a.zb;   // planes of this launch
    if (zn <= 0) return cudaErrorInvalidValue;
    dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (zn + a.zchunk - 1) / a.zchunk);
    a.ncta = grid.x * grid.y * grid.z;
    vti_sweep_kernel<RXY, RZ, TX, TY, LA>
        <<<grid, C::NT, C::SMEM, s>>>(tm.p, tm.q, tm.pp, tm.qp, tm.kx, tm.kn, tm.kz, a);
    return cudaGetLastError();
}

#define FD_VTI_CONFIGS(X)  \
    X(12, 8, 64, 8, 2)     \
    X(12, 8, 64, 8, 3)     \
    X(12, 8, 32, 16, 2)    \
    X(12, 8, 32, 32, 2)    \
    X(4, 4, 64, 8, 2)

cudaError_t launch_vti(int rxy, int rz, const Launch &L, const VtiMaps &tm, const VtiArgs &a, cudaStream_t s)
{
#define FD_VTI_CASE(RXY_, RZ_, TX_, TY_, LA_)                                           \
    if (rxy == RXY_ && rz == RZ_ && L.tx == TX_ && L.ty == TY_ && L.lookahead == LA_) \
        return launch_vt<RXY_, RZ_, TX_, TY_, LA_>(tm, a, s);
    FD_VTI_CONFIGS(FD_VTI_CASE)
#undef FD_VTI_CASE
    return cudaErrorInvalidConfiguration;
}

bool vti_config_built(int rxy, int rz, const Launch &L)
{
#define FD_VTI_BUILT(RXY_, RZ_, TX_, TY_, LA_) \
    if (rxy == RXY_ && rz == RZ_ && L.tx == TX_ && L.ty == TY_ && L.lookahead == LA_) return true;
    FD_VTI_CONFIGS(FD_VTI_BUILT)
#undef FD_VTI_BUILT
    return false;
}

Launch vti_default_launch(int rxy, int rz, int nx, int ny, int nz)
{
    (void)rxy;
    Launch L;
    // R_z = 8: 32 x 32 tiles, two rows per thread, q's z queues in tensor memory
    // (512^3: +1.3 to +5.2 % against the one-row 64 x 8 form in same-box comparisons)
    L.tx = rz == 8 ? 32 : 64;
    L.ty = rz == 8 ? 32 : 8;
    L.lookahead = 2;
    // two CTAs per SM, chunks of at most 64 planes; at 512^3, 8 chunks of 64 planes
    // (184.1 vs 180.9 Gpts/s for 7 of 74, interleaved in one process)
    L.zchunk = wave_zchunk(L, nx, ny, nz, (long)device_sm_count() * 2, 2 * rz, 64);
    return L;
}

bool vti_supported(int rxy, int rz) { return (rxy == 12 && rz == 8) || (rxy == 4 && rz == 4); }

}  // namespace fdk
