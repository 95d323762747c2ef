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
//     registers; the new levels overwrite the older ones in place.
// Compulsory HBM traffic: 36 bytes per point update (read p, q, p_prev, q_prev,
// kx, kn, kz; write p, q).
#include "fd_internal.h"
#include "launch_shape.h"
#include "ptx.cuh"

namespace fdk {

constexpr long long kVtiWaitLimit = 2000000000LL;   // ~1 s

template <int RXY, int RZ, int TX, int TY, int LA>
struct VtiCfg {
    static constexpr int NTX = TX / 4;
    static constexpr int NC = NTX * TY;
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
    static constexpr int SMEM = OFF_BAR + 8 * (2 * NA + 2 * NB) + 16;
    static constexpr int NW = 2 * RZ + 1;
    static_assert(TX % 4 == 0 && RXY % 4 == 0, "x alignment");
    static_assert(NC % 32 == 0, "whole consumer warps");
    static_assert((SLOT_A * 4) % 128 == 0 && (TILE * 4) % 128 == 0, "slot alignment");
    static_assert(SW <= 256 && SH <= 256, "TMA box limit");
};

template <int RXY, int RZ, int TX, int TY, int LA>
__global__ void __launch_bounds__((TX / 4) * TY + 32, 2)
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
    int *sh = reinterpret_cast<int *>(emptyB + C::NB);   // [0] n, [1] abort, [2..3] issue counts
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
    __syncthreads();
    const int n = sh[0];
    bool failed = false;

    if (tid >= C::NC) {
        // ------------------------------------------------------------ producer warp
        if (tid == C::NC) {
            const CUtensorMap *maps[7] = {&tm_p, &tm_q, &tm_pp, &tm_qp, &tm_kx, &tm_kn, &tm_kz};
            for (const CUtensorMap *m : maps) prefetch_tmap(m);
            int a_end = z0, b_end = z0;
            bool ok = true;
            for (int k = z0; ok && k < z1; ++k) {
                if (*sh_abort) break;
                const int u = k - z0;
                const int sa = u % C::NA, sb = u % C::NB;
                if (u >= C::NA && !mbar_wait_bounded(&emptyA[sa], ((u / C::NA) - 1) & 1, kVtiWaitLimit)) {
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(&fullA[sa], C::SLOT_A * 4);
                tma_load_3d(ringA + sa * C::SLOT_A, &tm_p, &fullA[sa], x0 - RXY, y0 - RXY, k);
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
                const float gyz = gyv * gz;
                const float pcu[4] = {pc.x, pc.y, pc.z, pc.w};
                const float qc[4] = {qq[RZ].x, qq[RZ].y, qq[RZ].z, qq[RZ].w};
                const float ppu[4] = {ppv.x, ppv.y, ppv.z, ppv.w};
                const float qpu[4] = {qpv.x, qpv.y, qpv.z, qpv.w};
                const float kxu[4] = {kxv.x, kxv.y, kxv.z, kxv.w};
                const float knu[4] = {knv.x, knv.y, knv.z, knv.w};
                const float kzu[4] = {kzv.x, kzv.y, kzv.z, kzv.w};
                const float gu[4] = {g4.x, g4.y, g4.z, g4.w};
                float op[4], oq[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float G = gu[e] * gyz;
                    const float zt = kzu[e] * dq[e];
                    op[e] = fmaf(kxu[e], hp[e], fmaf(2.f, pcu[e], -G * ppu[e])) + zt;
                    oq[e] = fmaf(knu[e], hp[e], fmaf(2.f, qc[e], -G * qpu[e])) + zt;
                }
                if (k == a.src.sz && gyi == a.src.sy && a.src.sx >= gxi && a.src.sx < gxi + 4 && n < a.src.len) {
                    const float sv = a.src.tab[n];
                    op[a.src.sx - gxi] += sv;
                    if (a.src.into_q) oq[a.src.sx - gxi] += sv;
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
                    const int ry = gyi - a.rec.ry0;
                    const int row = n - a.rec.t0;
                    if (ry >= 0 && ry % a.rec.rsy == 0 && ry / a.rec.rsy < a.rec.rny && row >= 0 &&
                        row < a.rec.cap) {
                        float *trow = a.rec.trace + (long long)row * a.rec.nrec +
                                      (long long)(ry / a.rec.rsy) * a.rec.rnx;
                        for (int e = 0; e < 4; ++e) {
                            const int rx = gxi + e - a.rec.rx0;
                            if (gxi + e < a.nx && rx >= 0 && rx % a.rec.rsx == 0 && rx / a.rec.rsx < a.rec.rnx)
                                trow[rx / a.rec.rsx] = op[e];
                        }
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < 2 * RZ; ++m) qq[m] = qq[m + 1];
        }
        if (!ok) {
            *sh_abort = 1;
            failed = true;
        }
    }

    if (__syncthreads_or(failed) && tid == C::NC) {
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
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(vti_sweep_kernel<RXY, RZ, TX, TY, LA>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
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
    L.tx = 64;
    L.ty = 8;
    L.lookahead = 2;
    // two CTAs per SM; at 512^3, 7 chunks of 74 planes (147.3 vs 142.5 Gpts/s for 4 of 128 on one box)
    L.zchunk = wave_zchunk(L, nx, ny, nz, (long)device_sm_count() * 2, 2 * rz);
    return L;
}

bool vti_supported(int rxy, int rz) { return (rxy == 12 && rz == 8) || (rxy == 4 && rz == 4); }

}  // namespace fdk
