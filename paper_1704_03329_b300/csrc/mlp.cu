// Learned structure classifier: MLP 30 -> 64 -> 64 -> 4 (ReLU, softmax),
// its training (forward/backward and weight gradients on the tcgen05
// tensor cores in mlp_tc.cu, fixed-order partial sums, AdamW) and the
// classification pipeline with exact-CNA fallback.
//
// Parameters are one FP32 vector (PPMD_MLP_NPARAM values):
//   mu[30] | isd[30] | W1[30][64] | b1[64] | W2[64][64] | b2[64] | W3[64][4] | b3[4]
// with x' = (x - mu) isd (input standardisation, fitted to the training
// features, not trained) and y = x' W + b (input-major weights).  Each call packs BF16 copies of
// the weights in the operand layouts the tensor cores read.
#include <cuda_bf16.h>
#include <math.h>

#include "analysis.cuh"
#include "mlp_layout.cuh"
#include "mlp_tc.cuh"

namespace ppmd {

static_assert(NPARAM == PPMD_MLP_NPARAM, "parameter count");

// Fixed-order sum of the per-block partials.
__global__ void k_sum_partials(const float *__restrict__ part, int nblk, float *__restrict__ grad) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NPARAM) return;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * NPARAM + e];
    grad[e] = s;
}

// AdamW (decoupled weight decay on the weight matrices only), step t >= 1.
__global__ void k_adamw(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v, const float *__restrict__ g,
                        float lr, float wd, float b1, float b2, float eps, float c1, float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NPARAM) return;
    if (e < OFF_W1) return;  // input standardisation: fitted, not trained
    const bool weight = (e < OFF_B1) || (e >= OFF_W2 && e < OFF_B2) || (e >= OFF_W3 && e < OFF_B3);
    const float gr = g[e];
    const float mm = b1 * m[e] + (1.0f - b1) * gr;
    const float vv = b2 * v[e] + (1.0f - b2) * gr * gr;
    m[e] = mm;
    v[e] = vv;
    float pe = p[e];
    if (weight) pe -= lr * wd * pe;
    pe -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    p[e] = pe;
}

__global__ void k_sum_loss(const double *part, int nblk, float *loss) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)sh[0];
}

// Input standardisation from n feature rows: per feature (thread f of 32)
// sums of x and x^2 over rows, compensated (Kahan) in FP32 per thread (FP64
// arithmetic is slow on this part), then in FP64 across threads and blocks;
// one partial per block.
__global__ void k_feat_stats(int64_t n, const __nv_bfloat16 *__restrict__ x, double *__restrict__ part) {
    __shared__ double sh[8][32][2];
    const int f = threadIdx.x & 31, rl = threadIdx.x >> 5;
    float a = 0.0f, ac = 0.0f, b = 0.0f, bc = 0.0f;  // sums and their compensations
    for (int64_t r = (int64_t)blockIdx.x * 8 + rl; r < n; r += (int64_t)gridDim.x * 8) {
        const float v = __bfloat162float(x[r * 32 + f]);
        const float y1 = v - ac, t1 = a + y1;
        ac = (t1 - a) - y1;
        a = t1;
        const float y2 = fmaf(v, v, -bc), t2 = b + y2;
        bc = (t2 - b) - y2;
        b = t2;
    }
    double s = (double)a - (double)ac, s2 = (double)b - (double)bc;
    sh[rl][f][0] = s;
    sh[rl][f][1] = s2;
    __syncthreads();
    if (rl == 0) {
        for (int q = 1; q < 8; ++q) {
            s += sh[q][f][0];
            s2 += sh[q][f][1];
        }
        part[(blockIdx.x * 32 + f) * 2] = s;
        part[(blockIdx.x * 32 + f) * 2 + 1] = s2;
    }
}

__global__ void k_feat_norm(const double *__restrict__ part, int nblk, int64_t n, float *__restrict__ p) {
    const int f = threadIdx.x;
    if (f >= 30) return;
    double s = 0.0, s2 = 0.0;
    for (int b = 0; b < nblk; ++b) {
        s += part[(b * 32 + f) * 2];
        s2 += part[(b * 32 + f) * 2 + 1];
    }
    const double mu = s / (double)n, var = fmax(s2 / (double)n - mu * mu, 0.0);
    p[OFF_MU + f] = (float)mu;
    p[OFF_ISD + f] = var > 1e-12 ? (float)(1.0 / sqrt(var)) : 1.0f;
}

}  // namespace ppmd

using namespace ppmd;

extern "C" int ppmd_mlp_forward(ppmd_ctx *ctx, const float *params, const uint16_t *x, int64_t n, float *logits) {
    if (!ctx || !params || n < 0 || (n > 0 && (!x || !logits))) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_mlp_forward: bad argument");
    cudaSetDevice(ctx->device);
    return mlp_infer_tc(ctx, n, (const __nv_bfloat16 *)x, params, logits, nullptr, nullptr, 0.0f, nullptr, nullptr);
}

extern "C" int ppmd_mlp_grad(ppmd_ctx *ctx, const float *params, const uint16_t *x, const int8_t *y, int64_t batch,
                             float *grad, float *loss) {
    if (!ctx || !params || batch < 1 || !x || !y || !grad) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_mlp_grad: bad argument");
    cudaSetDevice(ctx->device);
    const size_t rows = (size_t)batch;
    __nv_bfloat16 *act = (__nv_bfloat16 *)scratch(ctx, S_AUX1, sizeof(__nv_bfloat16) * rows * (4 * 64 + 8));
    if (!act) return PPMD_ERR_NOMEM;
    __nv_bfloat16 *H1 = act, *H2 = H1 + rows * 64, *D1 = H2 + rows * 64, *D2 = D1 + rows * 64, *D3 = D2 + rows * 64;
    const int fb_grid = (int)mlp_train_tc_blocks(batch);
    const int64_t chunk = mlp_wgrad_tc_chunk(batch);
    const int wg_grid = (int)((batch + chunk - 1) / chunk);
    double *lpart = (double *)scratch(ctx, S_AUX2, sizeof(double) * fb_grid + sizeof(float) * (size_t)wg_grid * NPARAM + 64);
    if (!lpart) return PPMD_ERR_NOMEM;
    float *wpart = (float *)(lpart + fb_grid);
    PPMD_TRY(mlp_train_tc(ctx, batch, (const __nv_bfloat16 *)x, y, params, H1, H2, D1, D2, D3, lpart));
    int64_t nblk = 0;
    PPMD_TRY(mlp_wgrad_tc(ctx, batch, (const __nv_bfloat16 *)x, H1, H2, D1, D2, D3, params, wpart, &nblk));
    PPMD_LAUNCH(ctx, k_sum_partials, div_up(NPARAM, 256), 256, 0, wpart, wg_grid, grad);
    if (loss) PPMD_LAUNCH(ctx, k_sum_loss, 1, 256, 0, lpart, fb_grid, loss);
    return check_launch(ctx, "ppmd_mlp_grad");
}

extern "C" int ppmd_mlp_fit_input_norm(ppmd_ctx *ctx, float *params, const uint16_t *x, int64_t n) {
    if (!ctx || !params || n < 1 || !x) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_mlp_fit_input_norm: bad argument");
    cudaSetDevice(ctx->device);
    const int nblk = 256;
    double *part = (double *)scratch(ctx, S_AUX2, sizeof(double) * nblk * 64);
    if (!part) return PPMD_ERR_NOMEM;
    PPMD_LAUNCH(ctx, k_feat_stats, nblk, 256, 0, n, (const __nv_bfloat16 *)x, part);
    PPMD_LAUNCH(ctx, k_feat_norm, 1, 32, 0, part, nblk, n, params);
    return check_launch(ctx, "ppmd_mlp_fit_input_norm");
}

extern "C" int ppmd_mlp_adamw(ppmd_ctx *ctx, float *params, float *m, float *v, const float *grad, int64_t step, float lr,
                              float wd, float beta1, float beta2, float eps) {
    if (!ctx || !params || !m || !v || !grad || step < 1) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_mlp_adamw: bad argument");
    cudaSetDevice(ctx->device);
    const float c1 = (float)(1.0 - pow((double)beta1, (double)step)), c2 = (float)(1.0 - pow((double)beta2, (double)step));
    PPMD_LAUNCH(ctx, k_adamw, div_up(NPARAM, 256), 256, 0, params, m, v, grad, lr, wd, beta1, beta2, eps, c1, c2);
    return check_launch(ctx, "ppmd_mlp_adamw");
}

extern "C" int ppmd_mlp_train_step(ppmd_ctx *ctx, float *params, float *m, float *v, int64_t step, const uint16_t *x,
                                   const int8_t *y, int64_t batch, float lr, float wd, float *loss) {
    float *grad = (float *)scratch(ctx, S_AUX0, sizeof(float) * NPARAM);
    if (!grad) return PPMD_ERR_NOMEM;
    PPMD_TRY(ppmd_mlp_grad(ctx, params, x, y, batch, grad, loss));
    return ppmd_mlp_adamw(ctx, params, m, v, grad, step, lr, wd, 0.9f, 0.999f, 1e-8f);
}

// ---------------------------------------------------------------------
// Classification pipeline: features, MLP class and confidence written in
// the caller's order, exact CNA over the low-confidence atoms written over
// their class.
// ---------------------------------------------------------------------
extern "C" int ppmd_classify_boxes(ppmd_ctx *ctx, int mode, const double *pos, int64_t nbox, const int64_t *atom_off,
                                   const ppmd_box *boxes, double r_feat, double r_cna, const float *params, float threshold,
                                   int8_t *label, float *confidence, int64_t *n_fallback) {
    if (!ctx) return PPMD_ERR_INVALID;
    PPMD_TRY(check_boxes(ctx, nbox, atom_off, boxes, "ppmd_classify"));
    const int64_t n = atom_off[nbox];
    if ((n > 0 && (!pos || !label)) || mode < 0 || mode > 2 || (mode == 1 && !params) ||
        (mode != 2 && !(r_cna > 0)) || (mode == 1 && !(r_feat >= r_cna)) || (mode == 2 && !(r_feat > 0)) ||
        (mode == 2 && !(threshold >= 0.0f)))
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_classify: bad argument");
    cudaSetDevice(ctx->device);
    if (mode == 0) {
        if (n_fallback) *n_fallback = n;
        return ppmd_analyze_boxes(ctx, pos, nbox, atom_off, boxes, 0.0, r_cna, nullptr, nullptr, nullptr, label);
    }
    const size_t nn = (size_t)(n > 0 ? n : 1);
    if (mode == 2) {
        // bond order within a tolerance: Q4, Q6 over r_feat, nearest table value
        float *q = (float *)scratch(ctx, S_TMP0, sizeof(float) * 2 * nn);
        if (!q) return PPMD_ERR_NOMEM;
        int32_t max_nbr = snapshot_capacity_boxes(nbox, atom_off, boxes, r_feat);
        for (int attempt = 0;; ++attempt) {
            Snapshot s;
            PPMD_TRY(sorted_snapshot_boxes(ctx, pos, nbox, atom_off, boxes, r_feat, max_nbr, s));
            PPMD_TRY(boa_launch(ctx, n, s.xq, s.pos, s.st, s.nbr, s.cnt, s.max_nbr, s.ld, r_feat, s.Lmax, s.perm, q, q + nn,
                                nullptr));
            PPMD_TRY(boa_tolerance_launch(ctx, n, q, q + nn, threshold, label, confidence));
            if (!n_fallback) return check_launch(ctx, "ppmd_classify");
            const int rc = end_pipeline(ctx, attempt, max_nbr);
            if (rc == PIPELINE_RETRY) continue;
            *n_fallback = 0;
            return rc;
        }
    }
    int32_t max_nbr = snapshot_capacity_boxes(nbox, atom_off, boxes, r_feat);
    for (int attempt = 0;; ++attempt) {
        Snapshot s;
        PPMD_TRY(sorted_snapshot_boxes(ctx, pos, nbox, atom_off, boxes, r_feat, max_nbr, s));
        __nv_bfloat16 *feat = (__nv_bfloat16 *)scratch(ctx, S_TMP0, sizeof(__nv_bfloat16) * 32 * nn);
        int32_t *fb = (int32_t *)scratch(ctx, S_AUX1, sizeof(int32_t) * nn);
        if (!feat || !fb) return PPMD_ERR_NOMEM;
        int32_t *nfb = ctx->d_status + 4;  // the fallback count, read back with the status
        PPMD_TRY(features_launch(ctx, n, s.xq, s.pos, s.st, s.nbr, s.cnt, s.max_nbr, s.ld, r_feat, r_cna, s.Lmax, nullptr,
                                 nullptr, feat));
        // MLP class and confidence of every atom, in the caller's order
        PPMD_TRY(mlp_infer_tc(ctx, n, feat, params, nullptr, label, confidence, threshold, fb, nfb, s.perm));
        // exact CNA for the low-confidence atoms (as many as the device
        // found), written over their MLP class
        PPMD_TRY(cna_subset_launch(ctx, n, nfb, fb, s.xq, s.pos, s.st, s.nbr, s.cnt, s.max_nbr, s.ld, r_cna, s.Lmax,
                                   s.perm, label));
        PPMD_TRY(check_launch(ctx, "ppmd_classify"));
        if (!n_fallback) return PPMD_OK;  // asynchronous: an overflow stays latched
        int32_t hfb = 0;
        const int rc = end_pipeline(ctx, attempt, max_nbr, &hfb);
        if (rc == PIPELINE_RETRY) continue;
        *n_fallback = hfb;
        return rc;
    }
}

extern "C" int ppmd_classify(ppmd_ctx *ctx, int mode, const double *pos, int64_t n, const ppmd_box *box, double r_feat,
                             double r_cna, const float *params, float threshold, int8_t *label, float *confidence,
                             int64_t *n_fallback) {
    if (!ctx || !box || n < 0) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_classify: bad argument");
    const int64_t off[2] = {0, n};
    return ppmd_classify_boxes(ctx, mode, pos, 1, off, box, r_feat, r_cna, params, threshold, label, confidence,
                               n_fallback);
}
