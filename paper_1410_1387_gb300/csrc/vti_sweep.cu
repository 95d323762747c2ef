// VTI sweep: one leapfrog step (Eq. 3) of the pseudo-acoustic system of
// Eqs. 1-2 with the symmetric x-y stencil of radius R_xy (Eq. 4) and the
// per-plane z stencil of radius R_z (Eq. 5), damping layer, source and
// receiver lattice fused in:
//   Hp = (d_xx + d_yy) p,  Dq = d_zz q (weights of plane k, dz absorbed)
//   p^{n+1} = G (2p - G p_prev + kx Hp + kz Dq + s)
//   q^{n+1} = G (2q - G q_prev + kn Hp + kz Dq [+ s])
// p needs only x-y neighbours and q only z neighbours (Sec. 1), so:
//   * plane k of p^n with an R_xy halo is staged in shared memory by TMA (ring of
//     LA + 1 planes, zero fill outside the grid = the zero halo);
//   * each thread keeps the 2 R_z + 1 z neighbours of its 4 q values in
//     registers, read with 128-bit loads one plane ahead;
//   * p_prev, q_prev and the three kappa arrays are streamed once, one plane
//     ahead, and the new levels overwrite the older ones in place.
// Compulsory HBM traffic: 36 bytes per point update (read p, q, p_prev, q_prev,
// kx, kn, kz; write p, q).
#include "fd_internal.h"
#include "ptx.cuh"

namespace fdk {

constexpr long long kVtiWaitLimit = 2000000000LL;

template <int RXY, int RZ, int TX, int TY, int LA>
struct VtiCfg {
    static constexpr int NTX = TX / 4;
    static constexpr int NT = NTX * TY;
    static constexpr int SW = TX + 2 * RXY;
    static constexpr int SH = TY + 2 * RXY;
    static constexpr int SLOT = SW * SH;
    static constexpr int NS = LA + 1;
    static constexpr int BAR_OFF = NS * SLOT * 4;
    static constexpr int SMEM = BAR_OFF + NS * 8 + 16;
    static constexpr int NW = 2 * RZ + 1;
    static_assert(TX % 4 == 0 && RXY % 4 == 0, "x alignment");
    static_assert((SLOT * 4) % 128 == 0, "slot alignment");
    static_assert(SW <= 256 && SH <= 256, "TMA box limit");
};

template <int RXY, int RZ, int TX, int TY, int LA>
__global__ void __launch_bounds__((TX / 4) * TY, 1)
    vti_sweep_kernel(const __grid_constant__ CUtensorMap tm, const VtiArgs a)
{
    using C = VtiCfg<RXY, RZ, TX, TY, LA>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + C::BAR_OFF);
    int *sh_n = reinterpret_cast<int *>(full + C::NS);

    const int tid = threadIdx.x;
    const int tx = tid % C::NTX, ty = tid / C::NTX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, a.nz);
    const int gxi = x0 + 4 * tx, gyi = y0 + ty;
    const bool act = (gyi < a.ny) && (gxi < a.nx);

    if (tid == 0) {
        prefetch_tmap(&tm);
        for (int s = 0; s < C::NS; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
        const int n = *reinterpret_cast<volatile int *>(&a.st->step);
        __threadfence();
        if (atomicAdd(&a.st->done, 1u) == a.ncta - 1) {
            a.st->done = 0;
            *reinterpret_cast<volatile int *>(&a.st->step) = n + 1;
            __threadfence();
        }
        *sh_n = n;
    }
    __syncthreads();
    const int n = *sh_n;

    int issued_end = z0;
    if (tid == 0) {
        const int last = min(z0 + C::NS, z1);
        for (int p = z0; p < last; ++p) {
            const int s = (p - z0) % C::NS;
            mbar_arrive_expect_tx(&full[s], C::SLOT * 4);
            tma_load_3d(ring + s * C::SLOT, &tm, &full[s], x0 - RXY, y0 - RXY, p);
        }
        issued_end = last;
    }

    const long long rowoff = (long long)gyi * a.pitch + gxi;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

    // q queue: qq[RZ + m] = my 4 q values of plane k + m
    float4 qq[2 * RZ + 1];
#pragma unroll
    for (int m = 0; m < 2 * RZ; ++m) {
        const int p = z0 - RZ + m;
        qq[m] = (act && p >= 0 && p < a.nz) ? ld_nc_na(a.q + p * a.plane + rowoff) : zero4;
    }
    float4 qa_n = zero4;                     // q of plane k + RZ, loaded one plane early
    float4 pp_n = zero4, qp_n = zero4, kx_n = zero4, kn_n = zero4, kz_n = zero4;
    float4 g4 = zero4;
    float gyv = 0.f;
    if (act) {
        if (z0 + RZ < a.nz) qa_n = ld_nc_na(a.q + (z0 + RZ) * a.plane + rowoff);
        pp_n = ld_cs(a.pprev + z0 * a.plane + rowoff);
        qp_n = ld_cs(a.qprev + z0 * a.plane + rowoff);
        kx_n = ld_nc_na(a.kx + z0 * a.plane + rowoff);
        kn_n = ld_nc_na(a.kn + z0 * a.plane + rowoff);
        kz_n = ld_nc_na(a.kz + z0 * a.plane + rowoff);
        g4 = *reinterpret_cast<const float4 *>(a.gx + gxi);
        gyv = a.gy[gyi];
    }

    bool ok = true, broke = false;
    for (int k = z0; k < z1; ++k) {
        qq[2 * RZ] = qa_n;
        const float4 pp = pp_n, qp = qp_n, kxv = kx_n, knv = kn_n, kzv = kz_n;
        if (act && k + 1 < z1) {
            if (k + 1 + RZ < a.nz) qa_n = ld_nc_na(a.q + (k + 1 + RZ) * a.plane + rowoff);
            else qa_n = zero4;
            pp_n = ld_cs(a.pprev + (k + 1) * a.plane + rowoff);
            qp_n = ld_cs(a.qprev + (k + 1) * a.plane + rowoff);
            kx_n = ld_nc_na(a.kx + (k + 1) * a.plane + rowoff);
            kn_n = ld_nc_na(a.kn + (k + 1) * a.plane + rowoff);
            kz_n = ld_nc_na(a.kz + (k + 1) * a.plane + rowoff);
        }

        // Dq: weights of plane k, l = -RZ..RZ in ascending order
        float dq[4] = {0.f, 0.f, 0.f, 0.f};
        const float *wr = a.ztab + (long long)k * C::NW;
#pragma unroll
        for (int m = 0; m < C::NW; ++m) {
            const float w = __ldg(wr + m);
            dq[0] = fmaf(w, qq[m].x, dq[0]);
            dq[1] = fmaf(w, qq[m].y, dq[1]);
            dq[2] = fmaf(w, qq[m].z, dq[2]);
            dq[3] = fmaf(w, qq[m].w, dq[3]);
        }

        const int u = k - z0;
        if (!mbar_wait_bounded(&full[u % C::NS], (u / C::NS) & 1, kVtiWaitLimit)) ok = false;
        const float *t = ring + (u % C::NS) * C::SLOT;

        // Hp from the staged plane: x window then y pairs
        float xw[4 + 2 * RXY];
        const float *rw = t + (ty + RXY) * C::SW + 4 * tx;
#pragma unroll
        for (int m = 0; m < (4 + 2 * RXY) / 4; ++m) {
            const float4 v = *reinterpret_cast<const float4 *>(rw + 4 * m);
            xw[4 * m + 0] = v.x; xw[4 * m + 1] = v.y; xw[4 * m + 2] = v.z; xw[4 * m + 3] = v.w;
        }
        float hp[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) hp[e] = a.w0 * xw[RXY + e];
#pragma unroll
        for (int l = 1; l <= RXY; ++l)
#pragma unroll
            for (int e = 0; e < 4; ++e) hp[e] = fmaf(a.wxy[l], xw[RXY + e + l] + xw[RXY + e - l], hp[e]);
#pragma unroll
        for (int l = 1; l <= RXY; ++l) {
            const float4 up = *reinterpret_cast<const float4 *>(t + (ty + RXY + l) * C::SW + RXY + 4 * tx);
            const float4 dn = *reinterpret_cast<const float4 *>(t + (ty + RXY - l) * C::SW + RXY + 4 * tx);
            hp[0] = fmaf(a.wxy[l], up.x + dn.x, hp[0]);
            hp[1] = fmaf(a.wxy[l], up.y + dn.y, hp[1]);
            hp[2] = fmaf(a.wxy[l], up.z + dn.z, hp[2]);
            hp[3] = fmaf(a.wxy[l], up.w + dn.w, hp[3]);
        }

        if (act) {
            const float gyz = gyv * a.gz[k];
            const float pc[4] = {xw[RXY], xw[RXY + 1], xw[RXY + 2], xw[RXY + 3]};
            const float qc[4] = {qq[RZ].x, qq[RZ].y, qq[RZ].z, qq[RZ].w};
            const float ppu[4] = {pp.x, pp.y, pp.z, pp.w};
            const float qpu[4] = {qp.x, qp.y, qp.z, qp.w};
            const float kxu[4] = {kxv.x, kxv.y, kxv.z, kxv.w};
            const float knu[4] = {knv.x, knv.y, knv.z, knv.w};
            const float kzu[4] = {kzv.x, kzv.y, kzv.z, kzv.w};
            const float gu[4] = {g4.x, g4.y, g4.z, g4.w};
            float op[4], oq[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float G = gu[e] * gyz;
                const float zt = kzu[e] * dq[e];
                op[e] = fmaf(kxu[e], hp[e], fmaf(2.f, pc[e], -G * ppu[e])) + zt;
                oq[e] = fmaf(knu[e], hp[e], fmaf(2.f, qc[e], -G * qpu[e])) + zt;
            }
            if (k == a.src.sz && gyi == a.src.sy && a.src.sx >= gxi && a.src.sx < gxi + 4 &&
                n < a.src.len) {
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
                        if (gxi + e < a.nx && rx >= 0 && rx % a.rec.rsx == 0 &&
                            rx / a.rec.rsx < a.rec.rnx)
                            trow[rx / a.rec.rsx] = op[e];
                    }
                }
            }
        }

#pragma unroll
        for (int m = 0; m < 2 * RZ; ++m) qq[m] = qq[m + 1];

        if (__syncthreads_or(!ok)) {
            broke = true;
            break;
        }
        if (tid == 0 && k + C::NS < z1) {
            fence_proxy_async_smem();
            const int p = k + C::NS;
            const int s = (p - z0) % C::NS;
            mbar_arrive_expect_tx(&full[s], C::SLOT * 4);
            tma_load_3d(ring + s * C::SLOT, &tm, &full[s], x0 - RXY, y0 - RXY, p);
            issued_end = p + 1;
        }
    }

    if (tid == 0 && broke) {
        atomicOr(&a.st->err, kErrTmaTimeout);
        atomicCAS(&a.st->err_info, 0,
                  1 + (int)(blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)));
        for (int p = max(z0, issued_end - C::NS); p < issued_end; ++p) {
            const int u = p - z0;
            mbar_wait_bounded(&full[u % C::NS], (u / C::NS) & 1, kVtiWaitLimit);
        }
    }
}

template <int RXY, int RZ, int TX, int TY, int LA>
static cudaError_t launch_vt(const Launch &L, const CUtensorMap &tm, const VtiArgs &a0,
                             cudaStream_t s)
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
    dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (a.nz + a.zchunk - 1) / a.zchunk);
    a.ncta = grid.x * grid.y * grid.z;
    vti_sweep_kernel<RXY, RZ, TX, TY, LA><<<grid, C::NT, C::SMEM, s>>>(tm, a);
    return cudaGetLastError();
}

#define FD_VTI_CASE(RXY_, RZ_, TX_, TY_, LA_)                                             \
    if (rxy == RXY_ && rz == RZ_ && L.tx == TX_ && L.ty == TY_ && L.lookahead == LA_)    \
        return launch_vt<RXY_, RZ_, TX_, TY_, LA_>(L, tm, a, s);

cudaError_t launch_vti(int rxy, int rz, const Launch &L, const CUtensorMap &tm, const VtiArgs &a,
                       cudaStream_t s)
{
    FD_VTI_CASE(12, 8, 64, 16, 2)
    FD_VTI_CASE(12, 8, 64, 8, 2)
    FD_VTI_CASE(4, 4, 64, 16, 2)
    return cudaErrorInvalidConfiguration;
}

int vti_smem_bytes(int rxy, const Launch &L)
{
    const int sw = L.tx + 2 * rxy, sh = L.ty + 2 * rxy, ns = L.lookahead + 1;
    return ns * sw * sh * 4 + ns * 8 + 16;
}

bool vti_supported(int rxy, int rz) { return (rxy == 12 && rz == 8) || (rxy == 4 && rz == 4); }

#define FD_VTI_BUILT(RXY_, RZ_, TX_, TY_, LA_) \
    if (rxy == RXY_ && rz == RZ_ && L.tx == TX_ && L.ty == TY_ && L.lookahead == LA_) return true;

bool vti_config_built(int rxy, int rz, const Launch &L)
{
    FD_VTI_BUILT(12, 8, 64, 16, 2)
    FD_VTI_BUILT(12, 8, 64, 8, 2)
    FD_VTI_BUILT(4, 4, 64, 16, 2)
    return false;
}

}  // namespace fdk
