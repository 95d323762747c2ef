// Isotropic sweep: one leapfrog step (Eq. 3) of v^2 (d_xx + d_yy + d_zz) u with
// the order-2R central stencil of Eq. 4 on every axis, the Cerjan damping layer,
// the Ricker source and the receiver lattice fused in.
//
// Design (2.5D plane sweep, after the shared-memory x-y tile plus z register
// queue that Sec. 3 describes, rebuilt for sm_103a):
//   * a CTA owns a TX x TY column of the grid and a chunk of z planes;
//   * plane k of u^n, with an R-cell halo in x and y, is staged in shared memory
//     by one TMA 3D tile load; loads outside the grid return zeros, which is the
//     zero halo of Sec. 1 at no cost.  A ring of R + LA + 1 staged planes keeps
//     LA planes in flight ahead of the one the queue needs next;
//   * each thread owns 4 consecutive x points (one float4) of one row and keeps
//     their 2R+1 z neighbours in registers; x and y neighbours come from the
//     staged plane (x as 1 + R/2 aligned float4 reads, y as 2R float4 reads);
//   * u^{n-1} and kappa are read once with 128-bit streaming loads one plane
//     ahead, and u^{n+1} is written in place over u^{n-1} (each point reads its
//     own older value before any thread writes it);
//   * the damping is applied in its deferred form G (2u - G u_prev + kappa Lu + s),
//     which equals multiplying both new levels by G after each step (Cerjan)
//     without rewriting u^n.
// Compulsory HBM traffic: 16 bytes per point update (read u^n, u^{n-1}, kappa;
// write u^{n+1}).
#include "fd_internal.h"
#include "ptx.cuh"

namespace fdk {

// ~1 s at the GB300's 2 GHz SM clock: far beyond any TMA latency.
constexpr long long kWaitLimit = 2000000000LL;

template <int R, int TX, int TY, int LA>
struct IsoCfg {
    static constexpr int NTX = TX / 4;          // threads per tile row
    static constexpr int NT = NTX * TY;         // threads per CTA
    static constexpr int SW = TX + 2 * R;       // staged row width (floats)
    static constexpr int SH = TY + 2 * R;       // staged rows
    static constexpr int SLOT = SW * SH;        // floats per staged plane
    static constexpr int NS = R + LA + 1;       // ring slots
    static constexpr int BAR_OFF = NS * SLOT * 4;
    static constexpr int SMEM = BAR_OFF + NS * 8 + 16;
    static_assert(TX % 4 == 0 && R % 4 == 0, "x alignment");
    static_assert((SLOT * 4) % 128 == 0, "slot alignment");
    static_assert(SW <= 256 && SH <= 256, "TMA box limit");
};

template <int R, int TX, int TY, int LA>
__global__ void __launch_bounds__((TX / 4) * TY, 2)
    iso_sweep_kernel(const __grid_constant__ CUtensorMap tm, const IsoArgs a)
{
    using C = IsoCfg<R, TX, TY, LA>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + C::BAR_OFF);
    int *sh_n = reinterpret_cast<int *>(full + C::NS);

    const int tid = threadIdx.x;
    const int tx = tid % C::NTX, ty = tid / C::NTX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, a.nz);
    const int zend = min(z1 + R, a.nz);             // staged planes: [z0, zend)
    const int gxi = x0 + 4 * tx, gyi = y0 + ty;
    const bool act = (gyi < a.ny) && (gxi < a.nx);

    if (tid == 0) {
        prefetch_tmap(&tm);
        for (int s = 0; s < C::NS; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
        // Time index of u^n: every CTA reads it, the last CTA to do so advances it.
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

    int issued_end = z0;                            // thread 0: planes [z0, issued_end) issued
    if (tid == 0) {
        const int last = min(z0 + C::NS, zend);
        for (int p = z0; p < last; ++p) {
            const int s = (p - z0) % C::NS;
            mbar_arrive_expect_tx(&full[s], C::SLOT * 4);
            tma_load_3d(ring + s * C::SLOT, &tm, &full[s], x0 - R, y0 - R, p);
        }
        issued_end = last;
    }

    bool ok = true;
    const long long rowoff = (long long)gyi * a.pitch + gxi;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

    // z queue: q[R + m] = my 4 values of plane k + m, m = -R..R.
    float4 q[2 * R + 1];
#pragma unroll
    for (int m = 0; m < R; ++m) {
        const int p = z0 - R + m;
        q[m] = (act && p >= 0) ? ld_nc_na(a.cur + p * a.plane + rowoff) : zero4;
    }
#pragma unroll
    for (int m = 0; m < R; ++m) {
        const int p = z0 + m;
        float4 v = zero4;
        if (p < zend) {
            const int u = p - z0;
            if (mbar_wait_bounded(&full[u % C::NS], (u / C::NS) & 1, kWaitLimit))
                v = *reinterpret_cast<const float4 *>(ring + (u % C::NS) * C::SLOT +
                                                      (ty + R) * C::SW + R + 4 * tx);
            else
                ok = false;
        }
        q[R + m] = v;
    }

    float4 pv_n = zero4, kv_n = zero4;
    float4 g4 = zero4;
    float gyv = 0.f;
    if (act) {
        pv_n = ld_cs(a.prev + z0 * a.plane + rowoff);
        kv_n = ld_nc_na(a.kappa + z0 * a.plane + rowoff);
        g4 = *reinterpret_cast<const float4 *>(a.gx + gxi);
        gyv = a.gy[gyi];
    }

    bool broke = false;
    for (int k = z0; k < z1; ++k) {
        // my values of plane k + R enter the queue
        {
            const int p = k + R;
            float4 v = zero4;
            if (p < zend) {
                const int u = p - z0;
                if (mbar_wait_bounded(&full[u % C::NS], (u / C::NS) & 1, kWaitLimit))
                    v = *reinterpret_cast<const float4 *>(ring + (u % C::NS) * C::SLOT +
                                                          (ty + R) * C::SW + R + 4 * tx);
                else
                    ok = false;
            }
            q[2 * R] = v;
        }

        const float4 pv = pv_n, kv = kv_n;
        if (act && k + 1 < z1) {
            pv_n = ld_cs(a.prev + (k + 1) * a.plane + rowoff);
            kv_n = ld_nc_na(a.kappa + (k + 1) * a.plane + rowoff);
        }

        const float *t = ring + ((k - z0) % C::NS) * C::SLOT;
        // x window: floats [4tx - R, 4tx + 4 + R) of my row of plane k
        float xw[4 + 2 * R];
        const float *rw = t + (ty + R) * C::SW + 4 * tx;
#pragma unroll
        for (int m = 0; m < (4 + 2 * R) / 4; ++m) {
            const float4 v = *reinterpret_cast<const float4 *>(rw + 4 * m);
            xw[4 * m + 0] = v.x; xw[4 * m + 1] = v.y; xw[4 * m + 2] = v.z; xw[4 * m + 3] = v.w;
        }
        float acc[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[e] = a.w0 * xw[R + e];
#pragma unroll
        for (int l = 1; l <= R; ++l)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[e] = fmaf(a.wxy[l], xw[R + e + l] + xw[R + e - l], acc[e]);
#pragma unroll
        for (int l = 1; l <= R; ++l) {
            const float4 up = *reinterpret_cast<const float4 *>(t + (ty + R + l) * C::SW + R + 4 * tx);
            const float4 dn = *reinterpret_cast<const float4 *>(t + (ty + R - l) * C::SW + R + 4 * tx);
            acc[0] = fmaf(a.wxy[l], up.x + dn.x, acc[0]);
            acc[1] = fmaf(a.wxy[l], up.y + dn.y, acc[1]);
            acc[2] = fmaf(a.wxy[l], up.z + dn.z, acc[2]);
            acc[3] = fmaf(a.wxy[l], up.w + dn.w, acc[3]);
        }
#pragma unroll
        for (int l = 1; l <= R; ++l) {
            acc[0] = fmaf(a.wz[l], q[R + l].x + q[R - l].x, acc[0]);
            acc[1] = fmaf(a.wz[l], q[R + l].y + q[R - l].y, acc[1]);
            acc[2] = fmaf(a.wz[l], q[R + l].z + q[R - l].z, acc[2]);
            acc[3] = fmaf(a.wz[l], q[R + l].w + q[R - l].w, acc[3]);
        }

        if (act) {
            const float gyz = gyv * a.gz[k];
            const float cu[4] = {xw[R], xw[R + 1], xw[R + 2], xw[R + 3]};
            const float pu[4] = {pv.x, pv.y, pv.z, pv.w};
            const float ku[4] = {kv.x, kv.y, kv.z, kv.w};
            const float gu[4] = {g4.x, g4.y, g4.z, g4.w};
            float o[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float G = gu[e] * gyz;
                o[e] = fmaf(ku[e], acc[e], fmaf(2.f, cu[e], -G * pu[e]));
            }
            if (k == a.src.sz && gyi == a.src.sy && a.src.sx >= gxi && a.src.sx < gxi + 4 &&
                n < a.src.len)
                o[a.src.sx - gxi] += a.src.tab[n];
#pragma unroll
            for (int e = 0; e < 4; ++e) o[e] *= gu[e] * gyz;

            float *dst = a.prev + k * a.plane + rowoff;
            if (gxi + 3 < a.nx) {
                st_cs(dst, make_float4(o[0], o[1], o[2], o[3]));
            } else {
                for (int e = 0; e < 4; ++e)
                    if (gxi + e < a.nx) dst[e] = o[e];
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
                            trow[rx / a.rec.rsx] = o[e];
                    }
                }
            }
        }

#pragma unroll
        for (int m = 0; m < 2 * R; ++m) q[m] = q[m + 1];

        // plane k leaves the ring; its slot takes plane k + NS
        if (__syncthreads_or(!ok)) {
            broke = true;
            break;
        }
        if (tid == 0 && k + C::NS < zend) {
            fence_proxy_async_smem();
            const int p = k + C::NS;
            const int s = (p - z0) % C::NS;
            mbar_arrive_expect_tx(&full[s], C::SLOT * 4);
            tma_load_3d(ring + s * C::SLOT, &tm, &full[s], x0 - R, y0 - R, p);
            issued_end = p + 1;
        }
    }

    if (tid == 0 && broke) {
        // A bounded wait gave up: record it, then wait (bounded) for the copies
        // still in flight so that none lands in shared memory after exit.
        atomicOr(&a.st->err, kErrTmaTimeout);
        atomicCAS(&a.st->err_info, 0,
                  1 + (int)(blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)));
        for (int p = max(z0, issued_end - C::NS); p < issued_end; ++p) {
            const int u = p - z0;
            mbar_wait_bounded(&full[u % C::NS], (u / C::NS) & 1, kWaitLimit);
        }
    }
}

// ---------------------------------------------------------------------------

template <int R, int TX, int TY, int LA>
static cudaError_t launch_t(const Launch &L, const CUtensorMap &tm, const IsoArgs &a0,
                            cudaStream_t s)
{
    using C = IsoCfg<R, TX, TY, LA>;
    static bool attr_set[64] = {};   // per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(iso_sweep_kernel<R, TX, TY, LA>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    IsoArgs a = a0;
    dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (a.nz + a.zchunk - 1) / a.zchunk);
    a.ncta = grid.x * grid.y * grid.z;
    iso_sweep_kernel<R, TX, TY, LA><<<grid, C::NT, C::SMEM, s>>>(tm, a);
    return cudaGetLastError();
}

#define FD_ISO_CASE(R_, TX_, TY_, LA_)                                               \
    if (R == R_ && L.tx == TX_ && L.ty == TY_ && L.lookahead == LA_)                 \
        return launch_t<R_, TX_, TY_, LA_>(L, tm, a, s);

cudaError_t launch_iso(int R, const Launch &L, const CUtensorMap &tm, const IsoArgs &a,
                       cudaStream_t s)
{
    FD_ISO_CASE(4, 64, 16, 2)
    FD_ISO_CASE(4, 64, 8, 2)
    FD_ISO_CASE(4, 128, 8, 2)
    FD_ISO_CASE(4, 32, 16, 2)
    FD_ISO_CASE(4, 64, 16, 3)
    FD_ISO_CASE(8, 64, 16, 2)
    FD_ISO_CASE(8, 64, 8, 2)
    FD_ISO_CASE(8, 32, 16, 2)
    return cudaErrorInvalidConfiguration;
}

int iso_smem_bytes(int R, const Launch &L)
{
    const int sw = L.tx + 2 * R, sh = L.ty + 2 * R, ns = R + L.lookahead + 1;
    return ns * sw * sh * 4 + ns * 8 + 16;
}

bool iso_supported(int R) { return R == 4 || R == 8; }

#define FD_ISO_BUILT(R_, TX_, TY_, LA_) \
    if (R == R_ && L.tx == TX_ && L.ty == TY_ && L.lookahead == LA_) return true;

bool iso_config_built(int R, const Launch &L)
{
    FD_ISO_BUILT(4, 64, 16, 2)
    FD_ISO_BUILT(4, 64, 8, 2)
    FD_ISO_BUILT(4, 128, 8, 2)
    FD_ISO_BUILT(4, 32, 16, 2)
    FD_ISO_BUILT(4, 64, 16, 3)
    FD_ISO_BUILT(8, 64, 16, 2)
    FD_ISO_BUILT(8, 64, 8, 2)
    FD_ISO_BUILT(8, 32, 16, 2)
    return false;
}

}  // namespace fdk
