// proposal.cu -- the learned candidate proposal: a small CNN that ranks the
// candidates of the relocalization grid from 176x47 gray views of the query
// and of the coarse-pose render, trained on the GPU with the kernels of
// gemm.cu (tcgen05 BF16 tensor cores, FP32 accumulation) and cnn.cu.
//
// Architecture (input NHWC [B][47][176][2]):
//   5 x { 3x3 conv, stride 2, pad 1, + bias, ReLU }: 2 -> 32 -> 64 -> 64 -> 128 -> 128
//   (spatial 47x176 -> 24x88 -> 12x44 -> 6x22 -> 3x11 -> 2x6)
//   flatten (NHWC order, 1536) -> FC 1024 + ReLU -> FC 64 (logits)
// Loss: softmax cross-entropy, mean over the batch; optimiser: Adam.
//
// Flat parameter layout (FP32, used for save/load and for checks): for each
// conv layer W[C_out][3][3][C_in] then b[C_out]; then FC1 W[1024][1536],
// b[1024]; FC2 W[64][1024], b[64] -- 1,916,960 values.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace reloc {

cudaError_t launch_downsample_gray(const float *img, int H, int W, int f, int ch, __nv_bfloat16 *out, cudaStream_t st);
cudaError_t launch_im2col(const __nv_bfloat16 *x, int B, int H, int W, int C, int Ho, int Wo, int Kp,
                          __nv_bfloat16 *col, cudaStream_t st);
cudaError_t launch_col2im(const float *dcol, int B, int H, int W, int C, int Ho, int Wo, int Kp, __nv_bfloat16 *dx_bf,
                          float *dx_f, cudaStream_t st);
cudaError_t launch_transpose_bf16(const __nv_bfloat16 *in, int R, int Cc, int ld_in, __nv_bfloat16 *out, int Rp, int Cp,
                                  cudaStream_t st, int ldo = 0);
cudaError_t launch_relu_back(const float *d, const __nv_bfloat16 *y, int64_t M, int N, __nv_bfloat16 *out,
                             cudaStream_t st);
cudaError_t launch_colsum(const __nv_bfloat16 *d, int R, int Cc, float *db, cudaStream_t st);
cudaError_t launch_softmax_ce(const float *logits, const int32_t *labels, int B, int C, float *loss_rows, float *dl,
                              __nv_bfloat16 *dlb, cudaStream_t st);
cudaError_t launch_adam(float *w, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2, float eps,
                        float c1, float c2, __nv_bfloat16 *w_bf, cudaStream_t st);
cudaError_t launch_to_bf16(const float *a, int64_t n, __nv_bfloat16 *b, cudaStream_t st);

namespace {

struct Conv {
    int Cin, Cout, H, W, Ho, Wo, K, Kp;
};

constexpr int IN_H = PROPOSAL_H, IN_W = PROPOSAL_W, IN_C = 2;
constexpr int FC1_IN = 1536, FC1_OUT = 1024, FC2_OUT = PROPOSAL_CLASSES;

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t n)
    {
        if (n <= bytes && p) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&p, n < 256 ? 256 : n);
        if (e == cudaSuccess) bytes = n < 256 ? 256 : n;
        return e;
    }
    ~Buf()
    {
        if (p) cudaFree(p);
    }
    template <typename T> T *as() const { return (T *)p; }
};

}  // namespace

struct ProposalNet {
    Conv conv[5];
    // parameter tensors (index: conv 0..4, fc1 5, fc2 6); weights padded [N][Kp]
    int wn[7], wk[7];            // rows, padded columns
    int64_t w_off[7], b_off[7];  // offsets into the FP32 master buffers
    int64_t n_master = 0;        // total FP32 master values (padded)
    Buf master, grad, m, v, wbf; // FP32 master params/grads/Adam state; BF16 weight copies
    int64_t wbf_off[7];
    int64_t steps = 0;
    // activations (sized for the largest batch seen)
    int cap_b = 0;
    Buf col[5], y[5], h1, logits, dl, dlb, loss_rows, tA, tB, dmid, dmid_bf, dcol, part, status;
};

int64_t proposal_param_count()
{
    int64_t n = 0;
    const int cin[5] = {2, 32, 64, 64, 128}, cout[5] = {32, 64, 64, 128, 128};
    for (int l = 0; l < 5; ++l) n += (int64_t)cout[l] * 9 * cin[l] + cout[l];
    n += (int64_t)FC1_OUT * FC1_IN + FC1_OUT + (int64_t)FC2_OUT * FC1_OUT + FC2_OUT;
    return n;
}

static int pad64(int k) { return (k + 63) / 64 * 64; }

ProposalNet *proposal_create(uint64_t seed, cudaError_t *err)
{
    ProposalNet *P = new ProposalNet();
    const int cin[5] = {2, 32, 64, 64, 128}, cout[5] = {32, 64, 64, 128, 128};
    int H = IN_H, W = IN_W;
    for (int l = 0; l < 5; ++l) {
        Conv &c = P->conv[l];
        c.Cin = cin[l];
        c.Cout = cout[l];
        c.H = H;
        c.W = W;
        c.Ho = (H - 1) / 2 + 1;
        c.Wo = (W - 1) / 2 + 1;
        c.K = 9 * cin[l];
        c.Kp = pad64(c.K);
        H = c.Ho;
        W = c.Wo;
        P->wn[l] = c.Cout;
        P->wk[l] = c.Kp;
    }
    P->wn[5] = FC1_OUT;
    P->wk[5] = FC1_IN;
    P->wn[6] = FC2_OUT;
    P->wk[6] = FC1_OUT;
    int64_t o = 0, ob = 0;
    for (int t = 0; t < 7; ++t) {
        P->w_off[t] = o;
        o += (int64_t)P->wn[t] * P->wk[t];
        P->b_off[t] = o;
        o += P->wn[t];
        P->wbf_off[t] = ob;
        ob += (int64_t)P->wn[t] * P->wk[t];
    }
    P->n_master = o;
    // He-normal init (std sqrt(2 / fan_in)), zero biases; SplitMix64 + Box-Muller
    std::vector<float> h(o, 0.f);
    uint64_t state = seed;
    auto next = [&]() {
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto uni = [&]() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
    for (int t = 0; t < 7; ++t) {
        const int fan_in = t < 5 ? P->conv[t].K : P->wk[t];
        const int kreal = t < 5 ? P->conv[t].K : P->wk[t];
        const double sd = std::sqrt(2.0 / fan_in);
        for (int r = 0; r < P->wn[t]; ++r)
            for (int k = 0; k < kreal; ++k) {
                const double u1 = uni(), u2 = uni();
                h[P->w_off[t] + (int64_t)r * P->wk[t] + k] =
                    (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
            }
    }
    cudaError_t e;
    if ((e = P->master.ensure(4 * o)) != cudaSuccess || (e = P->grad.ensure(4 * o)) != cudaSuccess ||
        (e = P->m.ensure(4 * o)) != cudaSuccess || (e = P->v.ensure(4 * o)) != cudaSuccess ||
        (e = P->wbf.ensure(2 * ob)) != cudaSuccess || (e = P->status.ensure(64)) != cudaSuccess) {
        *err = e;
        delete P;
        return nullptr;
    }
    cudaMemcpy(P->master.p, h.data(), 4 * o, cudaMemcpyHostToDevice);
    cudaMemset(P->grad.p, 0, 4 * o);
    cudaMemset(P->m.p, 0, 4 * o);
    cudaMemset(P->v.p, 0, 4 * o);
    cudaMemset(P->status.p, 0, 64);
    for (int t = 0; t < 7; ++t)
        launch_to_bf16(P->master.as<float>() + P->w_off[t], (int64_t)P->wn[t] * P->wk[t],
                       P->wbf.as<__nv_bfloat16>() + P->wbf_off[t], 0);
    *err = cudaDeviceSynchronize();
    if (*err != cudaSuccess) {
        delete P;
        return nullptr;
    }
    return P;
}

void proposal_destroy(ProposalNet *P) { delete P; }

// flat <-> padded master layout
static void flat_to_master(const ProposalNet *P, const float *flat, std::vector<float> &master)
{
    master.assign(P->n_master, 0.f);
    int64_t f = 0;
    for (int t = 0; t < 7; ++t) {
        const int kreal = t < 5 ? P->conv[t].K : P->wk[t];
        for (int r = 0; r < P->wn[t]; ++r)
            for (int k = 0; k < kreal; ++k) master[P->w_off[t] + (int64_t)r * P->wk[t] + k] = flat[f++];
        for (int r = 0; r < P->wn[t]; ++r) master[P->b_off[t] + r] = flat[f++];
    }
}

static void master_to_flat(const ProposalNet *P, const std::vector<float> &master, float *flat)
{
    int64_t f = 0;
    for (int t = 0; t < 7; ++t) {
        const int kreal = t < 5 ? P->conv[t].K : P->wk[t];
        for (int r = 0; r < P->wn[t]; ++r)
            for (int k = 0; k < kreal; ++k) flat[f++] = master[P->w_off[t] + (int64_t)r * P->wk[t] + k];
        for (int r = 0; r < P->wn[t]; ++r) flat[f++] = master[P->b_off[t] + r];
    }
}

cudaError_t proposal_get(const ProposalNet *P, int which, float *flat)
{
    std::vector<float> h(P->n_master);
    const Buf &b = which == 0 ? P->master : P->grad;
    cudaError_t e = cudaMemcpy(h.data(), b.p, 4 * P->n_master, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    master_to_flat(P, h, flat);
    return cudaSuccess;
}

cudaError_t proposal_set(ProposalNet *P, const float *flat)
{
    std::vector<float> h;
    flat_to_master(P, flat, h);
    cudaError_t e = cudaMemcpy(P->master.p, h.data(), 4 * P->n_master, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    cudaMemset(P->m.p, 0, 4 * P->n_master);
    cudaMemset(P->v.p, 0, 4 * P->n_master);
    P->steps = 0;
    for (int t = 0; t < 7; ++t)
        launch_to_bf16(P->master.as<float>() + P->w_off[t], (int64_t)P->wn[t] * P->wk[t],
                       P->wbf.as<__nv_bfloat16>() + P->wbf_off[t], 0);
    return cudaDeviceSynchronize();
}

static cudaError_t ensure_batch(ProposalNet *P, int B)
{
    if (B <= P->cap_b) return cudaSuccess;
    cudaError_t e;
    size_t max_col = 0, max_mid = 0, max_tr = 0;
    for (int l = 0; l < 5; ++l) {
        const Conv &c = P->conv[l];
        const size_t M = (size_t)B * c.Ho * c.Wo;
        if ((e = P->col[l].ensure(2 * M * c.Kp)) != cudaSuccess) return e;
        if ((e = P->y[l].ensure(2 * M * c.Cout)) != cudaSuccess) return e;
        max_col = std::max(max_col, M * c.Kp);
        max_mid = std::max(max_mid, M * c.Cout);
        max_tr = std::max(max_tr, M * (size_t)std::max(c.Kp, c.Cout));
    }
    max_mid = std::max(max_mid, (size_t)B * FC1_IN);
    max_tr = std::max(max_tr, (size_t)FC1_IN * FC1_OUT);
    max_tr = std::max(max_tr, (size_t)B * FC1_IN);
    if ((e = P->h1.ensure(2 * (size_t)B * FC1_OUT)) != cudaSuccess) return e;
    if ((e = P->logits.ensure(4 * (size_t)B * FC2_OUT)) != cudaSuccess) return e;
    if ((e = P->dl.ensure(4 * (size_t)B * FC2_OUT)) != cudaSuccess) return e;
    // backward signals are carried as hi | lo BF16 pairs: twice the columns
    if ((e = P->dlb.ensure(2 * 2 * (size_t)B * FC2_OUT)) != cudaSuccess) return e;
    if ((e = P->loss_rows.ensure(4 * (size_t)B)) != cudaSuccess) return e;
    if ((e = P->tA.ensure(2 * 2 * max_tr)) != cudaSuccess) return e;
    if ((e = P->tB.ensure(2 * 2 * max_tr)) != cudaSuccess) return e;
    if ((e = P->dmid.ensure(4 * std::max(max_mid, (size_t)B * FC1_OUT))) != cudaSuccess) return e;
    if ((e = P->dmid_bf.ensure(2 * 2 * std::max(max_mid, (size_t)B * FC1_OUT))) != cudaSuccess) return e;
    if ((e = P->dcol.ensure(4 * max_col)) != cudaSuccess) return e;
    if ((e = P->part.ensure(4 * (size_t)32 * 1024 * 1024)) != cudaSuccess) return e;   // split-K partials
    P->cap_b = B;
    return cudaSuccess;
}

#define PK(call)                                                                                                       \
    do {                                                                                                               \
        cudaError_t e_ = (call);                                                                                       \
        if (e_ != cudaSuccess) return e_;                                                                              \
    } while (0)

// Forward pass; logits FP32 [B][64] into P->logits (and out if given).
cudaError_t proposal_forward(ProposalNet *P, const __nv_bfloat16 *in, int B, float *out, cudaStream_t st)
{
    PK(ensure_batch(P, B));
    const __nv_bfloat16 *x = in;
    const __nv_bfloat16 *wbf = P->wbf.as<__nv_bfloat16>();
    const float *mst = P->master.as<float>();
    int *status = P->status.as<int>();
    for (int l = 0; l < 5; ++l) {
        const Conv &c = P->conv[l];
        const int M = B * c.Ho * c.Wo;
        PK(launch_im2col(x, B, c.H, c.W, c.Cin, c.Ho, c.Wo, c.Kp, P->col[l].as<__nv_bfloat16>(), st));
        PK(launch_gemm_bf16(P->col[l].as<__nv_bfloat16>(), wbf + P->wbf_off[l], mst + P->b_off[l], nullptr,
                            P->y[l].as<__nv_bfloat16>(), M, c.Cout, c.Kp, c.Kp, c.Kp, c.Cout, 1, 1, nullptr, status, st));
        x = P->y[l].as<__nv_bfloat16>();
    }
    PK(launch_gemm_bf16(x, wbf + P->wbf_off[5], mst + P->b_off[5], nullptr, P->h1.as<__nv_bfloat16>(), B, FC1_OUT,
                        FC1_IN, FC1_IN, FC1_IN, FC1_OUT, 1, 1, nullptr, status, st));
    PK(launch_gemm_bf16(P->h1.as<__nv_bfloat16>(), wbf + P->wbf_off[6], mst + P->b_off[6], out ? out : P->logits.as<float>(),
                        nullptr, B, FC2_OUT, FC1_OUT, FC1_OUT, FC1_OUT, FC2_OUT, 0, 1, nullptr, status, st));
    if (out) PK(cudaMemcpyAsync(P->logits.p, out, 4 * (size_t)B * FC2_OUT, cudaMemcpyDeviceToDevice, st));
    return cudaSuccess;
}

// largest divisor of k64 = K / 64 that is <= cap
static int split_for(int K, int cap)
{
    const int k64 = K / 64;
    for (int d = std::min(cap, k64); d >= 1; --d)
        if (k64 % d == 0) return d;
    return 1;
}

// Backward signals are carried as two BF16 terms, [M][2N] = hi | lo (x ~ hi +
// lo to ~16 significant bits), so the only BF16 rounding of the backward
// pass is that of the stored forward activations and weights.

// weight gradient gW[N][Kc] = dY^T X for the split dY [M][2N] and X [M][Kc]
// (BF16), M % 32 == 0: one GEMM over the 2M stacked rows, hi^T X + lo^T X
static cudaError_t weight_grad(ProposalNet *P, const __nv_bfloat16 *dY, int M, int N, const __nv_bfloat16 *X, int Kc,
                               float *gW, cudaStream_t st)
{
    __nv_bfloat16 *tA = P->tA.as<__nv_bfloat16>(), *tB = P->tB.as<__nv_bfloat16>();
    const int M2 = 2 * M;
    PK(launch_transpose_bf16(dY, M, N, 2 * N, tA, M, N, st, M2));          // [N][0, M): hi^T
    PK(launch_transpose_bf16(dY + N, M, N, 2 * N, tA + M, M, N, st, M2));  // [N][M, 2M): lo^T
    PK(launch_transpose_bf16(X, M, Kc, Kc, tB, M, Kc, st, M2));             // [Kc][2M]: X^T twice
    PK(launch_transpose_bf16(X, M, Kc, Kc, tB + M, M, Kc, st, M2));
    const int split = split_for(M2, std::max(1, (int)std::min<int64_t>(128, (int64_t)32 * 1024 * 1024 / ((int64_t)N * Kc))));
    return launch_gemm_bf16(tA, tB, nullptr, gW, nullptr, N, Kc, M2, M2, M2, Kc, 0, split, P->part.as<float>(),
                            P->status.as<int>(), st);
}

// input gradient dX[M][Kc] (FP32) = dY W for the split dY [M][2N] and the BF16
// weights W [N][Kc]: one GEMM over 2N, B = [W^T | W^T] ([Kc][2N])
static cudaError_t input_grad(ProposalNet *P, const __nv_bfloat16 *dY, int M, int N, const __nv_bfloat16 *W, int Kc,
                              float *dX, cudaStream_t st)
{
    __nv_bfloat16 *tB = P->tB.as<__nv_bfloat16>();
    PK(launch_transpose_bf16(W, N, Kc, Kc, tB, N, Kc, st, 2 * N));
    PK(launch_transpose_bf16(W, N, Kc, Kc, tB + N, N, Kc, st, 2 * N));
    return launch_gemm_bf16(dY, tB, nullptr, dX, nullptr, M, Kc, 2 * N, 2 * N, 2 * N, Kc, 0, 1, nullptr,
                            P->status.as<int>(), st);
}

// One training step on a batch (B % 64 == 0): forward, loss, backward; Adam
// update if `update`.  loss_dev: mean loss written as float.
cudaError_t proposal_train_step(ProposalNet *P, const __nv_bfloat16 *in, const int32_t *labels, int B, float lr,
                                bool update, float *loss_sum_dev, cudaStream_t st)
{
    PK(proposal_forward(P, in, B, nullptr, st));
    float *g = P->grad.as<float>();
    __nv_bfloat16 *wbf = P->wbf.as<__nv_bfloat16>();
    PK(launch_softmax_ce(P->logits.as<float>(), labels, B, FC2_OUT, P->loss_rows.as<float>(), P->dl.as<float>(),
                         P->dlb.as<__nv_bfloat16>(), st));
    if (loss_sum_dev) PK(cudaMemcpyAsync(loss_sum_dev, P->loss_rows.p, 4 * (size_t)B, cudaMemcpyDeviceToDevice, st));
    // FC2
    PK(weight_grad(P, P->dlb.as<__nv_bfloat16>(), B, FC2_OUT, P->h1.as<__nv_bfloat16>(), FC1_OUT, g + P->w_off[6], st));
    PK(launch_colsum(P->dlb.as<__nv_bfloat16>(), B, FC2_OUT, g + P->b_off[6], st));
    PK(input_grad(P, P->dlb.as<__nv_bfloat16>(), B, FC2_OUT, wbf + P->wbf_off[6], FC1_OUT, P->dmid.as<float>(), st));
    PK(launch_relu_back(P->dmid.as<float>(), P->h1.as<__nv_bfloat16>(), B, FC1_OUT, P->dmid_bf.as<__nv_bfloat16>(), st));
    // FC1
    const __nv_bfloat16 *x5 = P->y[4].as<__nv_bfloat16>();
    PK(weight_grad(P, P->dmid_bf.as<__nv_bfloat16>(), B, FC1_OUT, x5, FC1_IN, g + P->w_off[5], st));
    PK(launch_colsum(P->dmid_bf.as<__nv_bfloat16>(), B, FC1_OUT, g + P->b_off[5], st));
    PK(input_grad(P, P->dmid_bf.as<__nv_bfloat16>(), B, FC1_OUT, wbf + P->wbf_off[5], FC1_IN, P->dmid.as<float>(), st));
    // conv layers, last to first; dmid holds dL/dY_l (FP32, NHWC)
    for (int l = 4; l >= 0; --l) {
        const Conv &c = P->conv[l];
        const int M = B * c.Ho * c.Wo;
        PK(launch_relu_back(P->dmid.as<float>(), P->y[l].as<__nv_bfloat16>(), M, c.Cout,
                            P->dmid_bf.as<__nv_bfloat16>(), st));
        PK(weight_grad(P, P->dmid_bf.as<__nv_bfloat16>(), M, c.Cout, P->col[l].as<__nv_bfloat16>(), c.Kp,
                       g + P->w_off[l], st));
        PK(launch_colsum(P->dmid_bf.as<__nv_bfloat16>(), M, c.Cout, g + P->b_off[l], st));
        if (l == 0) break;
        PK(input_grad(P, P->dmid_bf.as<__nv_bfloat16>(), M, c.Cout, wbf + P->wbf_off[l], c.Kp, P->dcol.as<float>(), st));
        PK(launch_col2im(P->dcol.as<float>(), B, c.H, c.W, c.Cin, c.Ho, c.Wo, c.Kp, nullptr, P->dmid.as<float>(), st));
    }
    if (update) {
        P->steps++;
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float c1 = 1.f - std::pow(b1, (float)P->steps), c2 = 1.f - std::pow(b2, (float)P->steps);
        for (int t = 0; t < 7; ++t) {
            const int64_t nw = (int64_t)P->wn[t] * P->wk[t];
            PK(launch_adam(P->master.as<float>() + P->w_off[t], P->m.as<float>() + P->w_off[t],
                           P->v.as<float>() + P->w_off[t], g + P->w_off[t], nw, lr, b1, b2, eps, c1, c2,
                           wbf + P->wbf_off[t], st));
            PK(launch_adam(P->master.as<float>() + P->b_off[t], P->m.as<float>() + P->b_off[t],
                           P->v.as<float>() + P->b_off[t], g + P->b_off[t], P->wn[t], lr, b1, b2, eps, c1, c2, nullptr,
                           st));
        }
    }
    return cudaSuccess;
}

const float *proposal_logits(const ProposalNet *P) { return P->logits.as<float>(); }
int *proposal_status(const ProposalNet *P) { return P->status.as<int>(); }

cudaError_t proposal_make_input(const float *query, const float *seed_rgb, int H, int W, __nv_bfloat16 *out,
                                cudaStream_t st)
{
    const int f = H / IN_H;
    PK(launch_downsample_gray(query, H, W, f, 0, out, st));
    return launch_downsample_gray(seed_rgb, H, W, f, 1, out, st);
}

}  // namespace reloc
