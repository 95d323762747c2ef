// Small kernels around the sweep: model conversion (Sec. 1's velocities to the
// kappa arrays the step multiplies by), and the receiver gather for receiver
// sets that are not a lattice on one plane.
#include <math.h>

#include <algorithm>
#include <atomic>

#include <cudaTypedefs.h>

#include "fd_internal.h"

namespace fdk {

// cuTensorMapEncodeTiled through the runtime's driver entry-point lookup, so
// that the library links no libcuda and loads on machines without a GPU.
int encode_field_map(CUtensorMap *m, const float *base, int nx, int ny, int nz, long long pitch, int bx, int by)
{
    // the driver's encoder, looked up once (atomically: host threads may encode at once)
    static std::atomic<PFN_cuTensorMapEncodeTiled_v12000> enc_cache{nullptr};
    PFN_cuTensorMapEncodeTiled_v12000 enc = enc_cache.load(std::memory_order_acquire);
    if (!enc) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return (int)e;
        if (q != cudaDriverEntryPointSuccess || !fn) return -1;
        enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        enc_cache.store(enc, std::memory_order_release);
    }
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    cuuint64_t strides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)pitch * ny * 4};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return (int)r;
}

// Positive floats order like their bit patterns, so atomicMax on the bits is a
// float max for non-negative values.
__device__ __forceinline__ void atomic_max_pos(unsigned int *addr, float v)
{
    if (v > 0.f) atomicMax(addr, __float_as_uint(v));
}

__device__ __forceinline__ float warp_max(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ unsigned warp_sum(unsigned v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One block per (row j, plane k); threads stride over x.  `src_pitch` is nx for
// dense input or the field pitch when the input was copied in place.
__global__ void model_iso_kernel(const float *v, long long src_pitch, float *kappa, int nx,
                                 long long rows, long long pitch, double dt, DevState *st)
{
    float vmax = 0.f;
    unsigned bad = 0;
    // a block per row (j, k), rows taken in turn: ny * nz may exceed any grid dimension
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const float *vr = v + row * src_pitch;
        float *kr = kappa + row * pitch;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const float vv = vr[i];
            if (!(vv > 0.f) || !isfinite(vv)) ++bad;
            else vmax = fmaxf(vmax, vv);
            const double vd = (double)vv * dt;
            kr[i] = (float)(vd * vd);
        }
    }
    vmax = warp_max(vmax);
    bad = warp_sum(bad);
    if ((threadIdx.x & 31) == 0) {
        atomic_max_pos(reinterpret_cast<unsigned int *>(&st->vmax), vmax);
        if (bad) atomicAdd(&st->bad, bad);
    }
}

__global__ void model_vti_kernel(const float *vz, const float *eps, const float *delta,
                                 long long src_pitch, float *kx, float *kn, float *kz, int nx,
                                 long long rows, long long pitch, double dt, DevState *st)
{
    float vmax = 0.f, kxmax = 0.f;
    unsigned bad = 0, eld = 0;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const long long so = row * src_pitch;
    const long long dof = row * pitch;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const float v = vz[so + i], e = eps[so + i], d = delta[so + i];
        if (!(v > 0.f) || !isfinite(v) || !isfinite(e) || !isfinite(d) || !(1.0f + 2.0f * d > 0.f))
            ++bad;
        else
            vmax = fmaxf(vmax, v);
        if (e < d) ++eld;
        const double vd = (double)v * dt;
        const double k2 = vd * vd;
        const double kxd = k2 * (1.0 + 2.0 * (double)e);
        kz[dof + i] = (float)k2;
        kx[dof + i] = (float)kxd;
        kn[dof + i] = (float)(k2 * (1.0 + 2.0 * (double)d));
        if (isfinite(kxd)) kxmax = fmaxf(kxmax, (float)kxd);
    }
    }
    vmax = warp_max(vmax);
    kxmax = warp_max(kxmax);
    bad = warp_sum(bad);
    eld = warp_sum(eld);
    if ((threadIdx.x & 31) == 0) {
        atomic_max_pos(reinterpret_cast<unsigned int *>(&st->vmax), vmax);
        atomic_max_pos(reinterpret_cast<unsigned int *>(&st->kxmax), kxmax);
        if (bad) atomicAdd(&st->bad, bad);
        if (eld) atomicAdd(&st->eps_lt_delta, eld);
    }
}

// Receiver gather: after the step that made level n+1 (the time index on the
// device is then n+1), row n - t0 of the trace receives the field at idx.
__global__ void gather_kernel(const float *field, long long pitch, long long plane, const int *idx,
                              int nrec, float *trace, int t0, int cap, const DevState *st)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    const int row = *reinterpret_cast<const volatile int *>(&st->step) - 1 - t0;
    if (row < 0 || row >= cap) return;
    const int i = idx[3 * r], j = idx[3 * r + 1], k = idx[3 * r + 2];
    trace[(long long)row * nrec + r] = field[(long long)k * plane + (long long)j * pitch + i];
}

// Adjoint source rows and misfit: row m of inj = kappa(x_r) times the residual
// of step nt-1-m (the adjoint runs backward in time).
__global__ void adjoint_source_kernel(const RecLattice rec, const float *__restrict__ kappa, long long pitch,
                                      long long plane, const float *__restrict__ tr, const float *__restrict__ dobs,
                                      int nt, float *__restrict__ inj, double *misfit)
{
    const long long nrec = rec.nrec;
    const long long total = nrec * nt;
    double acc = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long n = t / nrec, r = t % nrec;
        const int x = rec.rx0 + (int)(r % rec.rnx) * rec.rsx, y = rec.ry0 + (int)(r / rec.rnx) * rec.rsy;
        const float d = tr[t] - dobs[t];
        acc += 0.5 * (double)d * (double)d;
        inj[(nt - 1 - n) * nrec + r] = kappa[(long long)rec.rk * plane + (long long)y * pitch + x] * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(misfit, acc);
}

cudaError_t launch_adjoint_source(const RecLattice &rec, const float *kappa, long long pitch, long long plane,
                                  const float *tr, const float *dobs, int nt, float *inj, double *misfit,
                                  cudaStream_t s)
{
    adjoint_source_kernel<<<4 * 152, 256, 0, s>>>(rec, kappa, pitch, plane, tr, dobs, nt, inj, misfit);
    return cudaGetLastError();
}

cudaError_t launch_model_iso(const float *v, long long src_pitch, float *kappa, int nx, int ny,
                             int nz, long long pitch, double dt, DevState *st, cudaStream_t s)
{
    const long long rows = (long long)ny * nz;
    model_iso_kernel<<<(unsigned)std::min<long long>(rows, 1 << 16), 128, 0, s>>>(v, src_pitch, kappa, nx, rows,
                                                                                   pitch, dt, st);
    return cudaGetLastError();
}

cudaError_t launch_model_vti(const float *vz, const float *eps, const float *delta,
                             long long src_pitch, float *kx, float *kn, float *kz, int nx, int ny,
                             int nz, long long pitch, double dt, DevState *st, cudaStream_t s)
{
    const long long rows = (long long)ny * nz;
    model_vti_kernel<<<(unsigned)std::min<long long>(rows, 1 << 16), 128, 0, s>>>(vz, eps, delta, src_pitch, kx, kn,
                                                                                   kz, nx, rows, pitch, dt, st);
    return cudaGetLastError();
}

cudaError_t launch_gather(const float *field, long long pitch, long long plane, const int *idx,
                          int nrec, float *trace, int t0, int cap, const DevState *st,
                          cudaStream_t s)
{
    if (nrec <= 0) return cudaSuccess;
    gather_kernel<<<(nrec + 255) / 256, 256, 0, s>>>(field, pitch, plane, idx, nrec, trace, t0, cap,
                                                     st);
    return cudaGetLastError();
}

}  // namespace fdk
