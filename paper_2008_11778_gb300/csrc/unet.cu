// unet.cu -- the learned preconditioner's network (a U-Net, not part of the
// paper) as a native runtime: parameters, activations, forward, backward and
// Adam, on the BF16 tensor-core GEMMs of unet_kernels.cu.
//
// Architecture (4 levels, base width C = 32):
//   enc l (l = 0..2): conv3x3(Cin -> C 2^l)+ReLU, conv3x3(-> C 2^l)+ReLU = skip_l, maxpool 2x2
//   bottom:           conv3x3(4C -> 8C)+ReLU, conv3x3(8C -> 8C)+ReLU
//   dec l (l = 2..0): upconv2x2 stride 2 (-> C 2^l, +bias), concat [up, skip_l],
//                     conv3x3(-> C 2^l)+ReLU, conv3x3(-> C 2^l)+ReLU
//   head:             conv1x1(C -> 1), FP32 output
// Input [B][2][H][W] FP32 (channel 0: gradient, 1: model, both normalised by
// the caller), output [B][H][W] FP32; H and W multiples of 8.
// Activations are NHWC BF16, every GEMM accumulates in FP32, parameters are
// FP32 masters with BF16 copies used by the kernels, Adam in FP32.
#include <cuda_bf16.h>

#include <climits>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/aafwi.h"
#include "internal.cuh"

namespace aafwi {

int unet_conv3_fwd(const __nv_bfloat16 *x, const __nv_bfloat16 *w, int B, int H, int W, int Cin, int Cout,
                   float *out, long long out_cap, cudaStream_t st);
int unet_conv3_dgrad(const __nv_bfloat16 *dz, const __nv_bfloat16 *wt, int B, int H, int W, int Cin, int Cout,
                     float *out, long long out_cap, cudaStream_t st);
int unet_conv3_wgrad(const __nv_bfloat16 *dz, const __nv_bfloat16 *x, int B, int H, int W, int Cin, int Cout,
                     int splits, float *out, cudaStream_t st);
int unet_up_fwd(const __nv_bfloat16 *x, const __nv_bfloat16 *w, int B, int H, int W, int Cin, int Cout,
                float *out, cudaStream_t st);
int unet_up_dgrad(const __nv_bfloat16 *dy, const __nv_bfloat16 *w, int B, int H, int W, int Cin, int Cout,
                  float *out, cudaStream_t st);
int unet_up_wgrad(const __nv_bfloat16 *x, const __nv_bfloat16 *dy, int B, int H, int W, int Cin, int Cout,
                  int splits, float *out, cudaStream_t st);

namespace {

typedef __nv_bfloat16 bf16;
constexpr int ET = 256;

inline int nblk(long long n) { return (int)std::min<long long>((n + ET - 1) / ET, 65535LL * 8); }

#define GRID_LOOP(i, n) for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// y = bf16(act(sum_splits out + bias)) for an [M][N] GEMM result
__global__ void k_epi(const float *out, int splits, long long MN, int N, const float *bias, int relu, bf16 *y)
{
    GRID_LOOP(i, MN) {
        float v = 0.f;
        for (int s = 0; s < splits; ++s) v += out[s * MN + i];
        v += bias[i % N];
        if (relu) v = fmaxf(v, 0.f);
        y[i] = __float2bfloat16_rn(v);
    }
}

// upconv epilogue: out [Pin][4][C] -> y [B][2H][2W][C] with bias
__global__ void k_epi_up(const float *out, int B, int H, int W, int C, const float *bias, bf16 *y)
{
    const long long n = (long long)B * H * W * 4 * C;
    GRID_LOOP(i, n) {
        const int c = (int)(i % C);
        const long long t = i / C;
        const int q = (int)(t % 4);
        const long long p = t / 4;
        const int x = (int)(p % W), yy = (int)((p / W) % H), b = (int)(p / ((long long)W * H));
        const long long dst = (((long long)b * 2 * H + 2 * yy + q / 2) * 2 * W + 2 * x + (q & 1)) * C + c;
        y[dst] = __float2bfloat16_rn(out[i] + bias[c]);
    }
}

// dz = bf16(sum_splits g) * (y > 0)   (ReLU backward on the post-activation y)
__global__ void k_relu_back(const float *g, int splits, long long n, const bf16 *y, bf16 *dz)
{
    GRID_LOOP(i, n) {
        float v = 0.f;
        for (int s = 0; s < splits; ++s) v += g[s * n + i];
        const bf16 vb = __float2bfloat16_rn(v);
        dz[i] = __bfloat162float(y[i]) > 0.f ? vb : __float2bfloat16_rn(0.f);
    }
}

// FP32 sum of split slices: dw = sum_splits parts  ([splits][n], fixed order; dw may be parts)
__global__ void k_sum_splits(const float *parts, int splits, long long n, float *dw)
{
    GRID_LOOP(i, n) {
        float v = 0.f;
        for (int s = 0; s < splits; ++s) v += parts[s * n + i];
        dw[i] = v;
    }
}

// bias gradient db[c] = sum_p dz[p][c]: one block per channel, fixed order
__global__ void k_bias_grad(const bf16 *dz, long long P, int C, float *db)
{
    __shared__ float sh[ET];
    const int c = blockIdx.x;
    float acc = 0.f;
    for (long long p = threadIdx.x; p < P; p += ET) acc += __bfloat162float(dz[p * C + c]);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = ET / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[c] = sh[0];
}

// bias gradient of an upconv from its fine-grid output gradient dy [Pfine][C]
// is the same reduction over the fine grid.

__global__ void k_maxpool(const bf16 *x, int B, int H, int W, int C, bf16 *y, unsigned char *arg)
{
    const long long n = (long long)B * (H / 2) * (W / 2) * C;
    GRID_LOOP(i, n) {
        const int c = (int)(i % C);
        const long long p = i / C;
        const int xo = (int)(p % (W / 2)), yo = (int)((p / (W / 2)) % (H / 2)), b = (int)(p / ((long long)(W / 2) * (H / 2)));
        float best = -INFINITY;
        int bi = 0;
        for (int q = 0; q < 4; ++q) {
            const float v = __bfloat162float(x[(((long long)b * H + 2 * yo + q / 2) * W + 2 * xo + (q & 1)) * C + c]);
            if (v > best) {
                best = v;
                bi = q;
            }
        }
        y[i] = __float2bfloat16_rn(best);
        arg[i] = (unsigned char)bi;
    }
}

// g_fine (FP32 accumulator, [B][H][W][C]) += scatter of dy (FP32) at the argmax
__global__ void k_maxpool_back(const float *dy, const unsigned char *arg, int B, int H, int W, int C, float *gx)
{
    const long long n = (long long)B * (H / 2) * (W / 2) * C;
    GRID_LOOP(i, n) {
        const int c = (int)(i % C);
        const long long p = i / C;
        const int xo = (int)(p % (W / 2)), yo = (int)((p / (W / 2)) % (H / 2)), b = (int)(p / ((long long)(W / 2) * (H / 2)));
        const int q = arg[i];
        gx[(((long long)b * H + 2 * yo + q / 2) * W + 2 * xo + (q & 1)) * C + c] += dy[i];
    }
}

// concat [P][Ca] ++ [P][Cb] -> [P][Ca+Cb]
__global__ void k_concat(const bf16 *a, int Ca, const bf16 *b, int Cb, long long P, bf16 *y)
{
    const int C = Ca + Cb;
    GRID_LOOP(i, P * C) {
        const long long p = i / C;
        const int c = (int)(i % C);
        y[i] = c < Ca ? a[p * Ca + c] : b[p * Cb + c - Ca];
    }
}

// split the FP32 gradient of a concat: first Ca channels -> ga (bf16), the rest added to gb (FP32)
__global__ void k_concat_back(const float *g, int Ca, int Cb, long long P, bf16 *ga, float *gb)
{
    const int C = Ca + Cb;
    GRID_LOOP(i, P * C) {
        const long long p = i / C;
        const int c = (int)(i % C);
        if (c < Ca) ga[p * Ca + c] = __float2bfloat16_rn(g[i]);
        else gb[p * Cb + c - Ca] += g[i];
    }
}

// w [Cout][9][Cin] -> wt [Cin][9][Cout]
__global__ void k_transpose_w(const bf16 *w, int Cout, int Cin, bf16 *wt)
{
    GRID_LOOP(i, (long long)Cout * 9 * Cin) {
        const int ci = (int)(i % Cin);
        const int tap = (int)((i / Cin) % 9);
        const int co = (int)(i / (9LL * Cin));
        wt[((long long)ci * 9 + tap) * Cout + co] = w[i];
    }
}

// input [B][2][H][W] FP32 (NCHW) -> [B][H][W][2] BF16
__global__ void k_pack_input(const float *x, int B, int H, int W, bf16 *y)
{
    const long long n = (long long)B * H * W;
    GRID_LOOP(i, n * 2) {
        const int c = (int)(i % 2);
        const long long p = i / 2;
        const long long hw = (long long)H * W;
        const long long b = p / hw, r = p - b * hw;
        y[i] = __float2bfloat16_rn(x[(b * 2 + c) * hw + r]);
    }
}

// head: out[p] = sum_c x[p][c] w[c] + b   (FP32)
__global__ void k_head(const bf16 *x, long long P, int C, const bf16 *w, const float *b, float *out)
{
    GRID_LOOP(p, P) {
        float acc = 0.f;
        for (int c = 0; c < C; ++c) acc += __bfloat162float(x[p * C + c]) * __bfloat162float(w[c]);
        out[p] = acc + b[0];
    }
}

// loss L = 1/(2P) sum (out - t)^2 (per-block partial sums), dout = (out - t)/P
__global__ void k_mse(const float *out, const float *t, long long P, float *dout, double *part)
{
    __shared__ double sh[ET];
    double acc = 0.0;
    GRID_LOOP(p, P) {
        const float d = out[p] - t[p];
        dout[p] = d / (float)P;
        acc += (double)d * d;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = ET / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_mse_finish(const double *part, int nb, long long P, double *loss)
{
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int i = 0; i < nb; ++i) a += part[i];
        *loss = 0.5 * a / (double)P;
    }
}

// head backward: gx[p][c] = dout[p] w[c] (FP32), dw[c] = sum_p dout[p] x[p][c], db = sum dout
__global__ void k_head_back_x(const float *dout, long long P, int C, const bf16 *w, float *gx)
{
    GRID_LOOP(i, P * C) {
        const long long p = i / C;
        const int c = (int)(i % C);
        gx[i] = dout[p] * __bfloat162float(w[c]);
    }
}

__global__ void k_head_back_w(const float *dout, const bf16 *x, long long P, int C, float *dw, float *db)
{
    __shared__ float sh[ET];
    const int c = blockIdx.x;   // c == C: bias
    float acc = 0.f;
    for (long long p = threadIdx.x; p < P; p += ET)
        acc += c < C ? dout[p] * __bfloat162float(x[p * C + c]) : dout[p];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = ET / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (c < C) dw[c] = sh[0];
        else db[0] = sh[0];
    }
}

// Adam on FP32 masters; writes the BF16 copies
__global__ void k_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2, bf16 *pb)
{
    GRID_LOOP(i, n) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        pb[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void k_to_bf16(const float *a, long long n, bf16 *b)
{
    GRID_LOOP(i, n) b[i] = __float2bfloat16_rn(a[i]);
}

// Learned-step features: stats = (max|g|, mean m, std m) in FP64 (one block),
// then x[0] = g / max|g|, x[1] = (m - mean) / std on the network grid
// [H][W] (zero outside the model's nz x nx corner).
__global__ void k_feat_stats(const float *g, const float *m, long long n, double *stats)
{
    __shared__ double s0[ET], s1[ET], s2[ET];
    double gm = 0.0, sm = 0.0, sq = 0.0;
    for (long long i = threadIdx.x; i < n; i += ET) {
        gm = fmax(gm, fabs((double)g[i]));
        sm += (double)m[i];
        sq += (double)m[i] * m[i];
    }
    s0[threadIdx.x] = gm;
    s1[threadIdx.x] = sm;
    s2[threadIdx.x] = sq;
    __syncthreads();
    for (int o = ET / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s0[threadIdx.x] = fmax(s0[threadIdx.x], s0[threadIdx.x + o]);
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mean = s1[0] / n;
        stats[0] = s0[0] > 0 ? s0[0] : 1.0;
        stats[1] = mean;
        const double var = s2[0] / n - mean * mean;
        stats[2] = var > 0 ? sqrt(var) : 1.0;
    }
}

__global__ void k_feat(const float *g, const float *m, int nz, int nx, int H, int W, const double *stats, float *x)
{
    const long long n = (long long)H * W;
    GRID_LOOP(i, n) {
        const int z = (int)(i / W), c = (int)(i % W);
        float a = 0.f, b = 0.f;
        if (z < nz && c < nx) {
            const long long j = (long long)z * nx + c;
            a = (float)(g[j] / stats[0]);
            b = (float)((m[j] - stats[1]) / stats[2]);
        }
        x[i] = a;
        x[n + i] = b;
    }
}

// out = clip(m + std_m * delta, lo, hi) on the model's nz x nx corner of [H][W]
__global__ void k_apply(const float *m, const float *delta, int nz, int nx, int W, const double *stats,
                        float lo, float hi, float *out)
{
    GRID_LOOP(i, (long long)nz * nx) {
        const int z = (int)(i / nx), c = (int)(i % nx);
        float v = (float)(m[i] + stats[2] * delta[(long long)z * W + c]);
        if (lo < hi) v = fminf(fmaxf(v, lo), hi);
        out[i] = v;
    }
}

// ---------------------------------------------------------------------------

struct Conv {
    int Cin, Cout;
    bool up;          // 2x2 stride-2 transposed conv (w [Cin][4][Cout]) else 3x3 (w [Cout][9][Cin])
    long long w, b;   // parameter offsets
    long long nw() const { return up ? 4LL * Cin * Cout : 9LL * Cin * Cout; }
};

}  // namespace
}  // namespace aafwi

using namespace aafwi;

struct aafwi_unet {
    int Bmax = 0, H = 0, W = 0, C = 32;
    std::vector<Conv> L;                  // 17 conv layers + head (index 17)
    long long nparam = 0, head_w = 0, head_b = 0;
    std::vector<void *> bufs;
    float *P = nullptr, *G = nullptr, *Mm = nullptr, *Vv = nullptr;  // masters, grads, Adam moments
    bf16 *Pb = nullptr, *Wt = nullptr;    // BF16 params, transposed 3x3 weights (dgrad)
    long long wt_size = 0;
    int adam_t = 0;
    // activations (BF16 NHWC) per level
    bf16 *xin = nullptr;
    bf16 *ea[3], *eb[3], *pool[3];        // enc conv a, conv b (skip), pooled
    unsigned char *arg[3];
    bf16 *ba = nullptr, *bb = nullptr;
    bf16 *up[3], *cat[3], *da[3], *db[3];
    float *out = nullptr, *dout = nullptr;
    // scratch
    float *gemm = nullptr;                // FP32 GEMM outputs [splits][M][N]
    long long gemm_size = 0;
    float *gacc = nullptr, *gacc2 = nullptr;   // FP32 activation-gradient accumulators
    bf16 *gb1 = nullptr, *gb2 = nullptr;       // BF16 activation gradients
    double *lpart = nullptr, *loss = nullptr;
    bool retired = false;   // a tensor-core wait ran out: every later call is refused
    std::string msg;
};

namespace {

int uerr(aafwi_unet *u, int code, const std::string &m)
{
    if (u) u->msg = m;
    set_call_error(m);
    return code;
}

// After a bounded tensor-core wait ran out, MMAs of the abandoned CTA may
// still have been in flight when it freed its tensor memory: the network is
// retired and refuses every later call.
constexpr const char *kUnetRetired =
    "a tensor-core wait ran out; the network is retired and refuses every later call: destroy it and "
    "reset the device context (cudaDeviceReset) before continuing";

int retire(aafwi_unet *u)
{
    u->retired = true;
    return uerr(u, AAFWI_ERR_TIMEOUT, kUnetRetired);
}

int refuse_retired(aafwi_unet *u)
{
    return u && u->retired ? uerr(u, AAFWI_ERR_TIMEOUT, kUnetRetired) : AAFWI_OK;
}

template <class T>
bool ualloc(aafwi_unet *u, T **p, size_t n)
{
    void *q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(n * sizeof(T), 16)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaMemset(q, 0, std::max<size_t>(n * sizeof(T), 16));
    u->bufs.push_back(q);
    *p = (T *)q;
    return true;
}

// level-l spatial size and channels
inline int Hl(const aafwi_unet *u, int l) { return u->H >> l; }
inline int Wl(const aafwi_unet *u, int l) { return u->W >> l; }
inline int Cl(const aafwi_unet *u, int l) { return u->C << l; }

const bf16 *wb(const aafwi_unet *u, const Conv &c) { return u->Pb + c.w; }

// forward of one 3x3 conv + bias + ReLU into y
void conv_fwd(aafwi_unet *u, const Conv &c, const bf16 *x, int B, int H, int W, bf16 *y, cudaStream_t st)
{
    const int s = unet_conv3_fwd(x, wb(u, c), B, H, W, c.Cin, c.Cout, u->gemm, u->gemm_size, st);
    const long long MN = (long long)B * H * W * c.Cout;
    count_launch();
    k_epi<<<nblk(MN), ET, 0, st>>>(u->gemm, s, MN, c.Cout, u->P + c.b, 1, y);
}

void up_fwd(aafwi_unet *u, const Conv &c, const bf16 *x, int B, int H, int W, bf16 *y, cudaStream_t st)
{
    unet_up_fwd(x, wb(u, c), B, H, W, c.Cin, c.Cout, u->gemm, st);
    count_launch();
    k_epi_up<<<nblk((long long)B * H * W * 4 * c.Cout), ET, 0, st>>>(u->gemm, B, H, W, c.Cout, u->P + c.b, y);
}

int wgrad_splits(long long P) { return (int)std::max<long long>(1, std::min<long long>(64, P / 2048)); }

// Backward of y = relu(conv3(x) + b): gy (FP32 [P][Cout]) -> dW, db (into u->G),
// returns gx in FP32 (u->gemm, its split slices summed into the first) when want_gx.
void conv_back(aafwi_unet *u, const Conv &c, const bf16 *x, const bf16 *y, const float *gy, int B, int H, int W,
               bool want_gx, cudaStream_t st)
{
    const long long P = (long long)B * H * W;
    count_launch(3);
    k_relu_back<<<nblk(P * c.Cout), ET, 0, st>>>(gy, 1, P * c.Cout, y, u->gb1);
    k_bias_grad<<<c.Cout, ET, 0, st>>>(u->gb1, P, c.Cout, u->G + c.b);
    const int s = unet_conv3_wgrad(u->gb1, x, B, H, W, c.Cin, c.Cout, wgrad_splits(P), u->gemm, st);
    k_sum_splits<<<nblk(c.nw()), ET, 0, st>>>(u->gemm, s, c.nw(), u->G + c.w);
    if (want_gx) {
        count_launch();
        bf16 *wt = u->Wt;
        k_transpose_w<<<nblk(c.nw()), ET, 0, st>>>(wb(u, c), c.Cout, c.Cin, wt);
        const int sx = unet_conv3_dgrad(u->gb1, wt, B, H, W, c.Cin, c.Cout, u->gemm, u->gemm_size, st);
        if (sx > 1) {   // sum the slices in place into the first
            count_launch();
            k_sum_splits<<<nblk(P * c.Cin), ET, 0, st>>>(u->gemm, sx, P * c.Cin, u->gemm);
        }
    }
}

// Backward of y = upconv(x) + b (no activation): gy (BF16 [B][2H][2W][Cout])
void up_back(aafwi_unet *u, const Conv &c, const bf16 *x, const bf16 *gy, int B, int H, int W, cudaStream_t st)
{
    const long long Pin = (long long)B * H * W;
    count_launch(2);
    k_bias_grad<<<c.Cout, ET, 0, st>>>(gy, 4 * Pin, c.Cout, u->G + c.b);
    const int s = unet_up_wgrad(x, gy, B, H, W, c.Cin, c.Cout, wgrad_splits(Pin), u->gemm, st);
    k_sum_splits<<<nblk(c.nw()), ET, 0, st>>>(u->gemm, s, c.nw(), u->G + c.w);
    unet_up_dgrad(gy, wb(u, c), B, H, W, c.Cin, c.Cout, u->gemm, st);
}

void forward(aafwi_unet *u, const float *xin, int B, cudaStream_t st)
{
    count_launch();
    k_pack_input<<<nblk((long long)B * u->H * u->W * 2), ET, 0, st>>>(xin, B, u->H, u->W, u->xin);
    const bf16 *x = u->xin;
    int li = 0;
    for (int l = 0; l < 3; ++l) {
        const int H = Hl(u, l), W = Wl(u, l);
        conv_fwd(u, u->L[li++], x, B, H, W, u->ea[l], st);
        conv_fwd(u, u->L[li++], u->ea[l], B, H, W, u->eb[l], st);
        count_launch();
        k_maxpool<<<nblk((long long)B * H / 2 * W / 2 * Cl(u, l)), ET, 0, st>>>(u->eb[l], B, H, W, Cl(u, l), u->pool[l], u->arg[l]);
        x = u->pool[l];
    }
    conv_fwd(u, u->L[li++], x, B, Hl(u, 3), Wl(u, 3), u->ba, st);
    conv_fwd(u, u->L[li++], u->ba, B, Hl(u, 3), Wl(u, 3), u->bb, st);
    x = u->bb;
    for (int l = 2; l >= 0; --l) {
        const int H = Hl(u, l), W = Wl(u, l);
        up_fwd(u, u->L[li++], x, B, H / 2, W / 2, u->up[l], st);
        const long long P = (long long)B * H * W;
        count_launch();
        k_concat<<<nblk(P * 2 * Cl(u, l)), ET, 0, st>>>(u->up[l], Cl(u, l), u->eb[l], Cl(u, l), P, u->cat[l]);
        conv_fwd(u, u->L[li++], u->cat[l], B, H, W, u->da[l], st);
        conv_fwd(u, u->L[li++], u->da[l], B, H, W, u->db[l], st);
        x = u->db[l];
    }
    const long long P = (long long)B * u->H * u->W;
    count_launch();
    k_head<<<nblk(P), ET, 0, st>>>(x, P, u->C, u->Pb + u->head_w, u->P + u->head_b, u->out);
}

// Backward from dout (FP32 [P]) into u->G.  Activation gradients are carried
// in FP32 (the dgrad GEMM output) and rounded to BF16 only where they become a
// GEMM operand (ReLU backward, the upconv output gradient).
void backward(aafwi_unet *u, int B, cudaStream_t st)
{
    const long long P0 = (long long)B * u->H * u->W;
    const int C = u->C;
    count_launch(2);
    k_head_back_w<<<C + 1, ET, 0, st>>>(u->dout, u->db[0], P0, C, u->G + u->head_w, u->G + u->head_b);
    k_head_back_x<<<nblk(P0 * C), ET, 0, st>>>(u->dout, P0, C, u->Pb + u->head_w, u->gacc);
    float *gskip[3];
    {
        long long off = 0;
        for (int l = 0; l < 3; ++l) {
            gskip[l] = u->gacc2 + off;
            off += (long long)B * Hl(u, l) * Wl(u, l) * Cl(u, l);
        }
    }
    const float *g = u->gacc;          // FP32 gradient of the current activation
    int li = 16;
    for (int l = 0; l <= 2; ++l) {     // decoder levels, finest first
        const int H = Hl(u, l), W = Wl(u, l), Cv = Cl(u, l);
        const long long P = (long long)B * H * W;
        conv_back(u, u->L[li--], u->da[l], u->db[l], g, B, H, W, true, st);   // dec b
        conv_back(u, u->L[li--], u->cat[l], u->da[l], u->gemm, B, H, W, true, st);   // dec a
        cudaMemsetAsync(gskip[l], 0, P * Cv * sizeof(float), st);
        count_launch();
        k_concat_back<<<nblk(P * 2 * Cv), ET, 0, st>>>(u->gemm, Cv, Cv, P, u->gb2, gskip[l]);
        const bf16 *xin = l == 2 ? u->bb : u->db[l + 1];
        up_back(u, u->L[li--], xin, u->gb2, B, H / 2, W / 2, st);               // upconv
        g = u->gemm;                   // gradient of the coarser level's output
    }
    // bottom (level 3): li == 7
    conv_back(u, u->L[li--], u->ba, u->bb, g, B, Hl(u, 3), Wl(u, 3), true, st);
    conv_back(u, u->L[li--], u->pool[2], u->ba, u->gemm, B, Hl(u, 3), Wl(u, 3), true, st);
    for (int l = 2; l >= 0; --l) {     // encoder levels, coarsest first
        const int H = Hl(u, l), W = Wl(u, l), Cv = Cl(u, l);
        count_launch();
        k_maxpool_back<<<nblk((long long)B * H / 2 * W / 2 * Cv), ET, 0, st>>>(u->gemm, u->arg[l], B, H, W, Cv,
                                                                                gskip[l]);
        conv_back(u, u->L[li--], u->ea[l], u->eb[l], gskip[l], B, H, W, true, st);          // enc b
        const bf16 *xin = l == 0 ? u->xin : u->pool[l - 1];
        conv_back(u, u->L[li--], xin, u->ea[l], u->gemm, B, H, W, l > 0, st);             // enc a
    }
}

void loss_and_grad(aafwi_unet *u, const float *xin, const float *target, int B, cudaStream_t st)
{
    forward(u, xin, B, st);
    const long long P = (long long)B * u->H * u->W;
    const int nb = (int)std::min<long long>(4096, (P + ET - 1) / ET);
    count_launch(2);
    k_mse<<<nb, ET, 0, st>>>(u->out, target, P, u->dout, u->lpart);
    k_mse_finish<<<1, 32, 0, st>>>(u->lpart, nb, P, u->loss);
    backward(u, B, st);
}

}  // namespace

extern "C" {

int aafwi_unet_create(int Bmax, int H, int W, int C, aafwi_unet **out)
{
    if (!out || Bmax < 1 || H < 8 || W < 8 || H % 8 || W % 8 || C < 8 || C % 8)
        return uerr(nullptr, AAFWI_ERR_ARG, "unet_create: need Bmax >= 1, H, W multiples of 8, C multiple of 8");
    *out = nullptr;
    auto *u = new aafwi_unet();
    u->Bmax = Bmax;
    u->H = H;
    u->W = W;
    u->C = C;
    long long off = 0;
    auto add = [&](int cin, int cout, bool up) {
        Conv c{cin, cout, up, 0, 0};
        c.w = off;
        off += c.nw();
        c.b = off;
        off += cout;
        u->L.push_back(c);
    };
    add(2, C, false);
    add(C, C, false);
    add(C, 2 * C, false);
    add(2 * C, 2 * C, false);
    add(2 * C, 4 * C, false);
    add(4 * C, 4 * C, false);
    add(4 * C, 8 * C, false);
    add(8 * C, 8 * C, false);
    for (int l = 2; l >= 0; --l) {
        add(C << (l + 1), C << l, true);
        add(C << (l + 1), C << l, false);
        add(C << l, C << l, false);
    }
    u->head_w = off;
    off += C;
    u->head_b = off;
    off += 1;
    u->nparam = off;
    long long maxw = 0;
    for (auto &c : u->L) maxw = std::max(maxw, c.nw());
    u->wt_size = maxw;
    const long long P0 = (long long)Bmax * H * W;
    // largest GEMM output: max over layers of M*N*splits
    long long gs = 0;
    for (int l = 0; l < 4; ++l) {
        const long long P = P0 >> (2 * l);
        gs = std::max(gs, P * (8LL * C) * 2);        // activations x widest channels (concat)
        gs = std::max(gs, (long long)wgrad_splits(P) * maxw);
    }
    u->gemm_size = gs;
    bool ok = ualloc(u, &u->P, off) && ualloc(u, &u->G, off) && ualloc(u, &u->Mm, off) && ualloc(u, &u->Vv, off) &&
              ualloc(u, &u->Pb, off) && ualloc(u, &u->Wt, maxw) && ualloc(u, &u->xin, P0 * 2) &&
              ualloc(u, &u->gemm, gs) && ualloc(u, &u->gacc, P0 * 8 * C) && ualloc(u, &u->gacc2, P0 * 2 * C) &&
              ualloc(u, &u->gb1, P0 * 8 * C) && ualloc(u, &u->gb2, P0 * 8 * C) && ualloc(u, &u->out, P0) &&
              ualloc(u, &u->dout, P0) && ualloc(u, &u->lpart, 4096) && ualloc(u, &u->loss, 1);
    for (int l = 0; l < 3 && ok; ++l) {
        const long long P = P0 >> (2 * l);
        const int Cv = C << l;
        ok = ualloc(u, &u->ea[l], P * Cv) && ualloc(u, &u->eb[l], P * Cv) && ualloc(u, &u->pool[l], P / 4 * Cv) &&
             ualloc(u, &u->arg[l], P / 4 * Cv) && ualloc(u, &u->up[l], P * Cv) && ualloc(u, &u->cat[l], P * 2 * Cv) &&
             ualloc(u, &u->da[l], P * Cv) && ualloc(u, &u->db[l], P * Cv);
    }
    ok = ok && ualloc(u, &u->ba, (P0 >> 6) * 8 * C) && ualloc(u, &u->bb, (P0 >> 6) * 8 * C);
    if (!ok) {
        for (void *p : u->bufs) cudaFree(p);
        delete u;
        return uerr(nullptr, AAFWI_ERR_NOMEM, "unet_create: cudaMalloc failed");
    }
    *out = u;
    return AAFWI_OK;
}

void aafwi_unet_destroy(aafwi_unet *u)
{
    if (!u) return;
    for (void *p : u->bufs) cudaFree(p);
    delete u;
}

long long aafwi_unet_param_count(const aafwi_unet *u) { return u ? u->nparam : 0; }

int aafwi_unet_set_params(aafwi_unet *u, const float *host, long long n)
{
    if (int rc0 = refuse_retired(u)) return rc0;
    if (!u || !host || n != u->nparam) return uerr(u, AAFWI_ERR_ARG, "unet_set_params: size mismatch");
    cudaError_t e = cudaMemcpy(u->P, host, n * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        count_launch();
        k_to_bf16<<<nblk(n), ET>>>(u->P, n, u->Pb);
        e = cudaMemset(u->Mm, 0, n * sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(u->Vv, 0, n * sizeof(float));
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    u->adam_t = 0;
    if (e != cudaSuccess) return uerr(u, AAFWI_ERR_CUDA, std::string("unet_set_params: ") + cudaGetErrorString(e));
    return AAFWI_OK;
}

int aafwi_unet_get_params(aafwi_unet *u, float *host, long long n)
{
    if (int rc0 = refuse_retired(u)) return rc0;
    if (!u || !host || n != u->nparam) return uerr(u, AAFWI_ERR_ARG, "unet_get_params: size mismatch");
    cudaError_t e = cudaMemcpy(host, u->P, n * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return uerr(u, AAFWI_ERR_CUDA, std::string("unet_get_params: ") + cudaGetErrorString(e));
    return AAFWI_OK;
}

int aafwi_unet_forward(aafwi_unet *u, const float *x, int B, float *y, aafwi_stream stream)
{
    if (int rc0 = refuse_retired(u)) return rc0;
    if (!u || !x || !y || B < 1 || B > u->Bmax) return uerr(u, AAFWI_ERR_ARG, "unet_forward: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    forward(u, x, B, st);
    cudaError_t e = cudaMemcpyAsync(y, u->out, (size_t)B * u->H * u->W * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return uerr(u, AAFWI_ERR_CUDA, std::string("unet_forward: ") + cudaGetErrorString(e));
    return AAFWI_OK;
}

int aafwi_unet_loss_grad(aafwi_unet *u, const float *x, const float *target, int B, float *grad,
                         double *loss_host, aafwi_stream stream)
{
    if (int rc0 = refuse_retired(u)) return rc0;
    if (!u || !x || !target || B < 1 || B > u->Bmax) return uerr(u, AAFWI_ERR_ARG, "unet_loss_grad: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    loss_and_grad(u, x, target, B, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && grad)
        e = cudaMemcpyAsync(grad, u->G, u->nparam * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && loss_host) {
        e = cudaMemcpyAsync(loss_host, u->loss, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && unet_take_error()) return retire(u);
    }
    if (e != cudaSuccess) return uerr(u, AAFWI_ERR_CUDA, std::string("unet_loss_grad: ") + cudaGetErrorString(e));
    return AAFWI_OK;
}

int aafwi_learned_features(const float *grad, const float *m, int nz, int nx, int H, int W, float *x,
                           double *stats, aafwi_stream stream)
{
    if (!grad || !m || !x || !stats || nz < 1 || nx < 1 || H < nz || W < nx)
        return uerr(nullptr, AAFWI_ERR_ARG, "learned_features: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    count_launch(2);
    k_feat_stats<<<1, ET, 0, st>>>(grad, m, (long long)nz * nx, stats);
    k_feat<<<nblk((long long)H * W), ET, 0, st>>>(grad, m, nz, nx, H, W, stats, x);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return uerr(nullptr, AAFWI_ERR_CUDA, cudaGetErrorString(e));
    return AAFWI_OK;
}

int aafwi_learned_apply(const float *m, const float *delta, int nz, int nx, int W, const double *stats, float lo,
                        float hi, float *out, aafwi_stream stream)
{
    if (!m || !delta || !stats || !out || nz < 1 || nx < 1 || W < nx)
        return uerr(nullptr, AAFWI_ERR_ARG, "learned_apply: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    count_launch();
    k_apply<<<nblk((long long)nz * nx), ET, 0, st>>>(m, delta, nz, nx, W, stats, lo, hi, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return uerr(nullptr, AAFWI_ERR_CUDA, cudaGetErrorString(e));
    return AAFWI_OK;
}

int aafwi_unet_train_step(aafwi_unet *u, const float *x, const float *target, int B, float lr,
                          double *loss_host, aafwi_stream stream)
{
    if (int rc0 = refuse_retired(u)) return rc0;
    int rc = aafwi_unet_loss_grad(u, x, target, B, nullptr, nullptr, stream);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    ++u->adam_t;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)u->adam_t), c2 = 1.f - std::pow(b2, (float)u->adam_t);
    count_launch();
    k_adam<<<nblk(u->nparam), ET, 0, st>>>(u->P, u->G, u->Mm, u->Vv, u->nparam, lr, b1, b2, 1e-8f, c1, c2, u->Pb);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && loss_host) {
        e = cudaMemcpyAsync(loss_host, u->loss, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && unet_take_error()) return retire(u);
    }
    if (e != cudaSuccess) return uerr(u, AAFWI_ERR_CUDA, std::string("unet_train_step: ") + cudaGetErrorString(e));
    return AAFWI_OK;
}

int aafwi_unet_conv3x3(int op, const void *a, const void *b, int B, int H, int W, int Cin, int Cout, int splits,
                       float *out, long long out_cap, int *splits_used, aafwi_stream stream)
{
    if (!a || !b || !out || B < 1 || H < 1 || W < 1 || Cin < 1 || Cout < 1 || op < AAFWI_CONV3_FWD ||
        op > AAFWI_CONV3_WGRAD || (long long)B * H * W > INT_MAX / 9)
        return uerr(nullptr, AAFWI_ERR_ARG, "unet_conv3x3: bad arguments");
    const long long P = (long long)B * H * W;
    const long long MN = op == AAFWI_CONV3_WGRAD ? 9LL * Cin * Cout : P * (op == AAFWI_CONV3_FWD ? Cout : Cin);
    if (out_cap < MN) return uerr(nullptr, AAFWI_ERR_ARG, "unet_conv3x3: out_cap below one result");
    cudaStream_t st = (cudaStream_t)stream;
    const auto *x = static_cast<const bf16 *>(a), *y = static_cast<const bf16 *>(b);
    int s = 1;
    if (op == AAFWI_CONV3_FWD) {
        const long long cap = splits > 0 ? std::min(out_cap, splits * MN) : out_cap;
        s = unet_conv3_fwd(x, y, B, H, W, Cin, Cout, out, cap, st);
    } else if (op == AAFWI_CONV3_DGRAD) {
        const long long cap = splits > 0 ? std::min(out_cap, splits * MN) : out_cap;
        s = unet_conv3_dgrad(x, y, B, H, W, Cin, Cout, out, cap, st);
    } else {
        const long long want = splits > 0 ? splits : wgrad_splits(P);
        s = unet_conv3_wgrad(x, y, B, H, W, Cin, Cout, (int)std::max(1LL, std::min(want, out_cap / MN)), out, st);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return uerr(nullptr, AAFWI_ERR_CUDA, std::string("unet_conv3x3: ") + cudaGetErrorString(e));
    if (unet_take_error())
        return uerr(nullptr, AAFWI_ERR_TIMEOUT,
                    "unet_conv3x3: a tensor-core wait ran out; reset the device context (cudaDeviceReset) before "
                    "continuing");
    if (splits_used) *splits_used = s;
    return AAFWI_OK;
}

}  // extern "C"
