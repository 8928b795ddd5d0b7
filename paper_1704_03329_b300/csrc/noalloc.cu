// Lennard-Jones forces for callers that may not allocate device memory.
//
// Some callers cannot call cudaMalloc or let a library do it on their
// behalf: applications whose device memory is owned entirely by a host
// framework (a fixed pool or caching allocator that must account for every
// byte), or latency-critical loops in which an allocation, with the device
// synchronisation cudaMalloc/cudaFree may imply, is not allowed.  This entry
// point gives them the force loop of ppmd_lj_forces without a context and
// without any allocation: its working memory (fixed-point positions, block
// partial sums, a status word) lives in one statically sized device array
// of this file, which every GPU that loads the library holds until exit.
#include <mutex>

#include "lj.cuh"
#include "neighbours.cuh"

namespace {

using namespace ppmd;

constexpr int64_t MAX_ATOMS = PPMD_NOALLOC_MAX_ATOMS;
constexpr size_t XQ_BYTES = sizeof(int4) * (size_t)MAX_ATOMS;
// per-block (U, W) partial sums: at most MAX_ATOMS * 8 lanes / 256 threads + 1 blocks
constexpr size_t PART_ROWS = (size_t)(MAX_ATOMS * 8 / 256 + 1);
constexpr size_t PART_BYTES = 2 * sizeof(double) * PART_ROWS;
constexpr size_t TOT_OFF = XQ_BYTES + PART_BYTES;        // 2 doubles: U, W
constexpr size_t STATUS_OFF = TOT_OFF + 2 * sizeof(double);  // int32 status + uint64 needed
constexpr size_t SCRATCH_BYTES = STATUS_OFF + 32;

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

// Device address of the array, looked up once per device (the host-side
// name of a __device__ array is not a device address).
constexpr int MAX_DEVICES = 64;
std::mutex g_lock;
void *g_addr[MAX_DEVICES] = {nullptr};

int scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= MAX_DEVICES) return PPMD_ERR_INVALID;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            fprintf(stderr, "ppmd_lj_forces_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
            return PPMD_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = (unsigned char *)g_addr[dev];
    return PPMD_OK;
}

}  // namespace

extern "C" int ppmd_lj_forces_noalloc(void *cuda_stream, const double *pos, int64_t n, const ppmd_box *box,
                                      const ppmd_lj_params *lj, const int32_t *nbr, const int32_t *nbr_count,
                                      int32_t max_nbr, ppmd_prec prec, double *force, double *e_atom,
                                      double *e_total, double *virial) {
    if (n > MAX_ATOMS) {
        fprintf(stderr, "ppmd_lj_forces_noalloc: %lld atoms exceed the static limit of %lld (PPMD_NOALLOC_MAX_ATOMS)\n",
                (long long)n, (long long)MAX_ATOMS);
        return PPMD_ERR_CAPACITY;
    }
    if (!box || !lj || n < 0 || max_nbr < 0 || (prec != PPMD_FP32 && prec != PPMD_FP64)) return PPMD_ERR_INVALID;
    if (n > 0 && (!pos || !nbr_count || !force || (max_nbr > 0 && !nbr))) return PPMD_ERR_INVALID;
    if (!(lj->rc > 0) || !(lj->sigma > 0)) return PPMD_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PPMD_ERR_CUDA;
    unsigned char *base = nullptr;
    PPMD_TRY(scratch_address(dev, &base));
    // A context on the stack: it carries the stream and points its status
    // words into the static array; it owns no memory.
    ppmd_ctx local;
    local.device = dev;
    local.stream = (cudaStream_t)cuda_stream;
    local.d_status = (int32_t *)(base + STATUS_OFF);
    local.d_needed = (unsigned long long *)(base + STATUS_OFF + 8);
    int4 *xq = (int4 *)base;
    double *partials = (double *)(base + XQ_BYTES);
    double *tot = (double *)(base + TOT_OFF);
    SegTable st;
    st.d = nullptr;
    st.nseg = 1;
    PPMD_TRY(make_seg(&local, st.one, box->L, 0.0, lj->rc));
    const double Lmax = fmax(box->L[0], fmax(box->L[1], box->L[2]));
    const LJConst c = make_ljconst(*lj, Lmax);
    // the status words are the only contents that must start at zero
    PPMD_TRY(cuda_check(&local, cudaMemsetAsync(local.d_status, 0, 16, local.stream), "memset"));
    PPMD_TRY(prep_fixed(&local, pos, n, st, nullptr, xq, nullptr));
    const bool totals = e_total || virial;
    const int64_t nb = lj_blocks(n);
    if ((size_t)nb > PART_ROWS) return PPMD_ERR_CAPACITY;
    PPMD_TRY(lj_launch(&local, n, xq, pos, st, c, nbr, nbr_count, max_nbr, prec, nullptr, force, e_atom,
                       totals ? partials : nullptr));
    if (totals) {
        PPMD_TRY(reduce_partials(&local, partials, nb, 2, tot));
        if (e_total)
            PPMD_TRY(cuda_check(&local, cudaMemcpyAsync(e_total, tot, 8, cudaMemcpyDeviceToDevice, local.stream), "copy"));
        if (virial)
            PPMD_TRY(cuda_check(&local, cudaMemcpyAsync(virial, tot + 1, 8, cudaMemcpyDeviceToDevice, local.stream), "copy"));
    }
    return PPMD_OK;
}
