/*
 * One isotropic shot through the C ABI of libfd.so alone (include/fd.h and
 * the CUDA runtime; no Python): the caller allocates the arena and the trace
 * buffer, sets a model with a vertical velocity gradient v = 1800 + 10 k m/s,
 * a Ricker source at the centre, an x line of receivers through the centre,
 * runs `steps` steps as CUDA graphs of 8 steps (the second half through
 * fd_run_to_host, whose streamed rows must equal the ones read back after), and
 * writes the traces (steps x n floats) and then u^n (n^3 floats) to `out`.
 *
 * usage: shot_abi n radius steps sponge_width dt out
 */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "fd.h"

static int check(int rc, const char *what)
{
    if (rc != FD_OK) {
        char msg[512];
        fd_last_error(msg, sizeof msg);
        fprintf(stderr, "%s failed (%d): %s\n", what, rc, msg);
        exit(1);
    }
    return rc;
}

static void check_cuda(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) {
        fprintf(stderr, "%s failed: %s\n", what, cudaGetErrorString(e));
        exit(1);
    }
}

int main(int argc, char **argv)
{
    if (argc != 7) {
        fprintf(stderr, "usage: %s n radius steps sponge_width dt out\n", argv[0]);
        return 2;
    }
    const int n = atoi(argv[1]), R = atoi(argv[2]), steps = atoi(argv[3]), nb = atoi(argv[4]);
    const double dt = atof(argv[5]);

    fd_desc d = {0};
    d.mode = FD_MODE_ISO;
    d.nx = d.ny = d.nz = n;
    d.r_xy = d.r_z = R;
    d.h = d.dz = 10.0;
    d.dt = dt;
    d.sponge_width = nb;
    d.sponge_a = nb > 0 ? 0.015 : 0.0;

    cudaStream_t stream;
    check_cuda(cudaStreamCreate(&stream), "stream");
    size_t bytes = 0;
    check(fd_required_bytes(&d, &bytes), "fd_required_bytes");
    void *arena = NULL;
    check_cuda(cudaMalloc(&arena, bytes), "arena");
    fd_grid_t *g = NULL;
    check(fd_create_grid(&d, arena, bytes, stream, &g), "fd_create_grid");

    float *v = (float *)malloc(sizeof(float) * (size_t)n * n * n);
    for (int k = 0; k < n; ++k)
        for (size_t i = 0; i < (size_t)n * n; ++i) v[(size_t)k * n * n + i] = 1800.0f + 10.0f * (float)k;
    check(fd_set_model(g, v, NULL, NULL, FD_PTR_HOST), "fd_set_model");
    check(fd_add_source(g, n / 2, n / 2, n / 2, 15.0, 1.0 / 15.0, 1.0, 0), "fd_add_source");

    int *idx = (int *)malloc(sizeof(int) * 3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        idx[3 * i] = i;
        idx[3 * i + 1] = n / 2;
        idx[3 * i + 2] = n / 2;
    }
    float *trace_dev = NULL;
    check_cuda(cudaMalloc((void **)&trace_dev, sizeof(float) * (size_t)steps * n), "traces");
    check(fd_set_receivers(g, idx, n, trace_dev, steps), "fd_set_receivers");
    check(fd_set_graph(g, 8), "fd_set_graph");
    /* the first half by fd_run, the rest with its rows streamed to pinned host memory */
    const int half = steps / 2;
    check(fd_run(g, half), "fd_run");
    float *streamed = NULL;
    check_cuda(cudaMallocHost((void **)&streamed, sizeof(float) * (size_t)(steps - half) * n), "pinned rows");
    check(fd_run_to_host(g, steps - half, streamed, 0), "fd_run_to_host");

    float *tr = (float *)malloc(sizeof(float) * (size_t)steps * n);
    float *u = (float *)malloc(sizeof(float) * (size_t)n * n * n);
    check(fd_read_receivers(g, 0, steps, tr, FD_PTR_HOST), "fd_read_receivers");
    for (size_t i = 0; i < (size_t)(steps - half) * n; ++i)
        if (streamed[i] != tr[(size_t)half * n + i]) {
            fprintf(stderr, "streamed row value %zu differs from the read-back one\n", i);
            return 1;
        }
    check_cuda(cudaFreeHost(streamed), "free pinned rows");
    int tn = -1;
    check(fd_get_state(g, u, NULL, NULL, NULL, FD_PTR_HOST, &tn), "fd_get_state");
    if (tn != steps) {
        fprintf(stderr, "time index %d after %d steps\n", tn, steps);
        return 1;
    }
    check(fd_sync(g), "fd_sync");

    FILE *f = fopen(argv[6], "wb");
    if (!f || fwrite(tr, sizeof(float), (size_t)steps * n, f) != (size_t)steps * n ||
        fwrite(u, sizeof(float), (size_t)n * n * n, f) != (size_t)n * n * n) {
        fprintf(stderr, "cannot write %s\n", argv[6]);
        return 1;
    }
    fclose(f);

    check(fd_destroy_grid(g), "fd_destroy_grid");
    check_cuda(cudaFree(trace_dev), "free traces");
    check_cuda(cudaFree(arena), "free arena");
    check_cuda(cudaStreamDestroy(stream), "stream destroy");
    free(v);
    free(idx);
    free(tr);
    free(u);
    printf("ok\n");
    return 0;
}
