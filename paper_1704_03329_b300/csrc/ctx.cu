// Context, scratch memory, error latching, segment set-up, scans and
// fixed-order reductions.
#include <math.h>
#include <stdarg.h>

#include "common.cuh"

namespace ppmd {

int set_error(ppmd_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_check(ppmd_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return PPMD_OK;
    cudaGetLastError();  // reported here: not again by the next unrelated check
    return set_error(ctx, PPMD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int check_launch(ppmd_ctx *ctx, const char *what) { return cuda_check(ctx, cudaGetLastError(), what); }

void *scratch(ppmd_ctx *ctx, int slot, size_t bytes) {
    Scratch &s = ctx->scratch[slot];
    if (bytes == 0) bytes = 16;
    if (s.bytes >= bytes) return s.ptr;
    if (s.ptr) {
        // the stream may still use the old buffer
        cudaStreamSynchronize(ctx->stream);
        cudaFree(s.ptr);
        s.ptr = nullptr;
        s.bytes = 0;
    }
    size_t want = bytes + bytes / 8;
    if (cudaMalloc(&s.ptr, want) != cudaSuccess) {
        cudaGetLastError();
        set_error(ctx, PPMD_ERR_NOMEM, "cudaMalloc of %zu bytes failed", want);
        s.ptr = nullptr;
        return nullptr;
    }
    s.bytes = want;
    return s.ptr;
}

void *stage_host(ppmd_ctx *ctx, size_t bytes) {
    if (ctx->stage_ev) cudaEventSynchronize(ctx->stage_ev);
    if (bytes == 0) bytes = 16;
    if (ctx->h_stage_bytes >= bytes) return ctx->h_stage;
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    ctx->h_stage = nullptr;
    ctx->h_stage_bytes = 0;
    const size_t want = bytes + bytes / 4;
    if (cudaMallocHost(&ctx->h_stage, want) != cudaSuccess) {
        cudaGetLastError();
        set_error(ctx, PPMD_ERR_NOMEM, "cudaMallocHost of %zu bytes failed", want);
        ctx->h_stage = nullptr;
        return nullptr;
    }
    ctx->h_stage_bytes = want;
    return ctx->h_stage;
}

int stage_done(ppmd_ctx *ctx) {
    if (!ctx->stage_ev)
        PPMD_TRY(cuda_check(ctx, cudaEventCreateWithFlags(&ctx->stage_ev, cudaEventDisableTiming), "cudaEventCreate"));
    return cuda_check(ctx, cudaEventRecord(ctx->stage_ev, ctx->stream), "cudaEventRecord");
}

void cutoff_band(double rc2, double Lmax, float *lo, float *hi) {
    // The single-precision r^2 from fixed-point coordinates differs from
    // the exact value by at most ~6 units of 2^-24 relative plus the
    // quantisation of the two positions (L / 2^32 each); the band is a wide
    // multiple of that bound.
    double rc = sqrt(rc2);
    double band = 2e-5 * rc2 + 16.0 * rc * Lmax / 4294967296.0;
    *lo = (float)(rc2 - band);
    *hi = (float)(rc2 + band);
}

int make_seg(ppmd_ctx *ctx, Seg &s, const double L[3], double min_cell_width, double r_list) {
    memset(&s, 0, sizeof(s));
    double Lmax = 0;
    for (int d = 0; d < 3; ++d) {
        if (!(L[d] > 0) || !isfinite(L[d])) return set_error(ctx, PPMD_ERR_INVALID, "box edge %d is %g", d, L[d]);
        s.L[d] = L[d];
        s.inv_L[d] = 1.0 / L[d];
        s.fxs[d] = 4294967296.0 / L[d];
        s.sx[d] = (float)(L[d] / 4294967296.0);
        if (min_cell_width > 0) {
            double nc = floor(L[d] / min_cell_width);
            if (nc < 3) return set_error(ctx, PPMD_ERR_BOX, "box edge %g holds fewer than 3 cells of width %g", L[d], min_cell_width);
            if (nc > 1 << 20) return set_error(ctx, PPMD_ERR_BOX, "too many cells along edge %d", d);
            s.nc[d] = (int32_t)nc;
            s.w[d] = L[d] / nc;
            s.inv_w[d] = 1.0 / s.w[d];
        } else {
            s.nc[d] = 1;
            s.w[d] = L[d];
            s.inv_w[d] = 1.0 / L[d];
        }
        if (L[d] > Lmax) Lmax = L[d];
    }
    if (r_list > 0) {
        for (int d = 0; d < 3; ++d)
            if (!(r_list < 0.5 * L[d])) return set_error(ctx, PPMD_ERR_BOX, "cutoff %g is not below half the box edge %g", r_list, L[d]);
        s.rl2 = r_list * r_list;
        cutoff_band(s.rl2, Lmax, &s.rl2_lo, &s.rl2_hi);
    }
    return PPMD_OK;
}

// ---------------------------------------------------------------------
// Exclusive scan (two levels, 4096 items per block).
// ---------------------------------------------------------------------
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *total) {
    __shared__ int32_t warp_tot[32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        int32_t t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;
    }
    __syncthreads();
    int32_t base = wid > 0 ? warp_tot[wid - 1] : 0;
    *total = warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
    return base + x - v;
}

__global__ void k_scan_tiles(const int32_t *in, int32_t *out, int64_t n, int32_t *tile_sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int32_t tot;
    int32_t ex = block_exclusive_scan(s, &tot);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_add(int32_t *out, int64_t n, const int32_t *tile_offsets) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t add = tile_offsets[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < n) out[base + k] += add;
}

__global__ void k_write_total(int32_t *out, int64_t n, const int32_t *tile_sums, int ntiles, const int32_t *tile_offsets) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        out[n] = ntiles > 0 ? tile_offsets[ntiles - 1] + tile_sums[ntiles - 1] : 0;
    }
}

int exclusive_scan(ppmd_ctx *ctx, const int32_t *in, int32_t *out, int64_t n) {
    int ntiles = div_up(n, SCAN_TILE);
    if (ntiles > SCAN_TILE) return set_error(ctx, PPMD_ERR_CAPACITY, "scan of %lld items exceeds %d", (long long)n, SCAN_TILE * SCAN_TILE);
    int32_t *sums = (int32_t *)scratch(ctx, S_SCAN, sizeof(int32_t) * (size_t)(2 * SCAN_TILE + 2));
    if (!sums) return PPMD_ERR_NOMEM;
    int32_t *offs = sums + SCAN_TILE + 1;
    if (ntiles > 0) PPMD_LAUNCH(ctx, k_scan_tiles, ntiles, SCAN_THREADS, 0, in, out, n, sums);
    if (ntiles > 1) {
        PPMD_LAUNCH(ctx, k_scan_tiles, 1, SCAN_THREADS, 0, sums, offs, (int64_t)ntiles, sums + SCAN_TILE);
        PPMD_LAUNCH(ctx, k_scan_add, ntiles, SCAN_THREADS, 0, out, n, offs);
        PPMD_LAUNCH(ctx, k_write_total, 1, 32, 0, out, n, sums, ntiles, offs);
    } else {
        cudaMemsetAsync(offs, 0, sizeof(int32_t), ctx->stream);
        PPMD_LAUNCH(ctx, k_write_total, 1, 32, 0, out, n, sums, ntiles, offs);
    }
    return check_launch(ctx, "exclusive_scan");
}

// ---------------------------------------------------------------------
// Fixed-order reduction of per-block FP64 partial sums.
// ---------------------------------------------------------------------
// Column c of the partial rows: thread t sums rows t, t + 256, ... in that
// order, then a fixed tree over the threads.  The columns (at most four)
// are summed in the same pass over the rows, so the loads of a row are in
// flight together.
__global__ void k_reduce_partials(const double *parts, int64_t nparts, int width, double *dst) {
    __shared__ double sh[256];
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t p = threadIdx.x; p < nparts; p += blockDim.x) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (c < width) s[c] += parts[p * width + c];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (c >= width) break;
        sh[threadIdx.x] = s[c];
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) dst[c] = sh[0];
        __syncthreads();
    }
}

int reduce_partials(ppmd_ctx *ctx, const double *parts, int64_t nparts, int width, double *dst) {
    if (width < 1 || width > 4) return set_error(ctx, PPMD_ERR_INVALID, "reduce_partials: width %d", width);
    PPMD_LAUNCH(ctx, k_reduce_partials, 1, 256, 0, parts, nparts, width, dst);
    return check_launch(ctx, "reduce_partials");
}

}  // namespace ppmd

using namespace ppmd;

extern "C" int ppmd_create(ppmd_ctx **out, int device, void *cuda_stream) {
    if (!out) return PPMD_ERR_INVALID;
    *out = nullptr;
    ppmd_ctx *ctx = new (std::nothrow) ppmd_ctx();
    if (!ctx) return PPMD_ERR_NOMEM;
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    int rc = cuda_check(ctx, cudaSetDevice(device), "cudaSetDevice");
    if (rc == PPMD_OK) {
        void *p = scratch(ctx, S_STATUS, 64);
        if (!p) rc = PPMD_ERR_NOMEM;
        else {
            ctx->d_status = (int32_t *)p;
            ctx->d_needed = (unsigned long long *)((char *)p + 8);
            rc = cuda_check(ctx, cudaMemset(p, 0, 64), "cudaMemset");
        }
    }
    if (rc == PPMD_OK) {
        void *h = nullptr;
        rc = cuda_check(ctx, cudaMallocHost(&h, 64), "cudaMallocHost");
        if (rc == PPMD_OK) {
            memset(h, 0, 64);
            ctx->h_status = (int32_t *)h;
            ctx->h_needed = (unsigned long long *)((char *)h + 8);
        }
    }
    if (rc != PPMD_OK) {
        fprintf(stderr, "ppmd_create: %s\n", ctx->err);
        ppmd_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return PPMD_OK;
}

extern "C" int ppmd_destroy(ppmd_ctx *ctx) {
    if (!ctx) return PPMD_OK;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    for (int s = 0; s < S_NSLOTS; ++s)
        if (ctx->scratch[s].ptr) cudaFree(ctx->scratch[s].ptr);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    if (ctx->stage_ev) cudaEventDestroy(ctx->stage_ev);
    delete ctx;
    return PPMD_OK;
}

extern "C" int ppmd_set_stream(ppmd_ctx *ctx, void *cuda_stream) {
    if (!ctx) return PPMD_ERR_INVALID;
    ctx->stream = (cudaStream_t)cuda_stream;
    return PPMD_OK;
}

namespace ppmd {
int status_sync(ppmd_ctx *ctx, int64_t *needed, int32_t *aux) {
    if (!ctx) return PPMD_ERR_INVALID;
    cudaSetDevice(ctx->device);
    int rc = cuda_check(ctx, cudaMemcpyAsync(ctx->h_status, ctx->d_status, aux ? 24 : 16, cudaMemcpyDeviceToHost,
                                             ctx->stream),
                        "status copy");
    if (rc == PPMD_OK) rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    if (rc != PPMD_OK) return rc;
    if (aux) *aux = ctx->h_status[4];
    int32_t st = ctx->h_status[0];
    int64_t nd = (int64_t)ctx->h_needed[0];
    if (ctx->host_needed > nd) nd = ctx->host_needed;
    if (needed) *needed = nd;
    ctx->host_needed = 0;
    if (st != 0) {
        cudaMemsetAsync(ctx->d_status, 0, 16, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        if (st < 0 && ctx->err[0] == 0) set_error(ctx, st, "device reported status %d", st);
        if (st == PPMD_ERR_CAPACITY)
            set_error(ctx, st, "capacity exceeded: %lld needed", (long long)nd);
    }
    return st;
}
}  // namespace ppmd

extern "C" int ppmd_status(ppmd_ctx *ctx, int64_t *needed) { return status_sync(ctx, needed, nullptr); }

extern "C" int ppmd_sync(ppmd_ctx *ctx) { return ppmd_status(ctx, nullptr); }

extern "C" const char *ppmd_last_error(const ppmd_ctx *ctx) { return ctx ? ctx->err : "null context"; }

extern "C" int64_t ppmd_kernel_count(const ppmd_ctx *ctx) { return ctx ? ctx->launches : 0; }
