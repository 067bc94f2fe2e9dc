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
                   const float *bias, __nv_bfloat16 *y, float *out, long long out_cap, cudaStream_t st);
int unet_conv3_dgrad(const __nv_bfloat16 *dz, const __nv_bfloat16 *wt, int B, int H, int W, int Cin, int Cout,
                     float *out, long long out_cap, cudaStream_t st);
int unet_conv3_wgrad(const __nv_bfloat16 *dz, const __nv_bfloat16 *x, int B, int H, int W, int Cin, int Cout,
                     int max_splits, float *out, cudaStream_t st);
int unet_up_fwd(const __nv_bfloat16 *x, const __nv_bfloat16 *wt, int B, int H, int W, int Cin, int Cout,
                float *out, cudaStream_t st);
int unet_up_dgrad(const __nv_bfloat16 *dy, const __nv_bfloat16 *w, int B, int H, int W, int Cin, int Cout,
                  float *out, cudaStream_t st);
int unet_up_wgrad(const __nv_bfloat16 *x, const __nv_bfloat16 *dy, int B, int H, int W, int Cin, int Cout,
                  int max_splits, float *out, cudaStream_t st);

namespace {

typedef __nv_bfloat16 bf16;
constexpr int ET = 256;
// The 2-channel network input is stored with XIN_C channels (the rest zero),
// so that the first 3x3 layer runs the windowed tensor-core GEMMs too.
constexpr int XIN_C = 16;

inline int nblk(long long n) { return (int)std::min<long long>((n + ET - 1) / ET, 65535LL * 8); }

#define GRID_LOOP(i, n) for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// The elementwise kernels work in chunks of 8 channels (every channel count of
// the network is a multiple of 8): a thread moves 16 bytes of BF16 or 32 bytes
// of FP32, with 32-bit index arithmetic (element counts below 2^31).  Each
// element's arithmetic is the same as element by element.
__device__ __forceinline__ void load8(const float *p, float (&v)[8])
{
    const float4 a = *reinterpret_cast<const float4 *>(p), b = *reinterpret_cast<const float4 *>(p + 4);
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
}

__device__ __forceinline__ uint4 bf16x8(const float (&v)[8])
{
    unsigned h[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) h[j] = __bfloat16_as_ushort(__float2bfloat16_rn(v[j]));
    return make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
}

// y = bf16(act(sum_splits out + bias)) over [MN] = [M][N], MN = 8 n8
__global__ void k_epi(const float *out, int splits, int n8, int N, const float *bias, int relu, bf16 *y)
{
    const long long MN = 8LL * n8;
    GRID_LOOP(i, n8) {
        const int e = 8 * (int)i, c = e % N;
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int s = 0; s < splits; ++s) {
            float u[8];
            load8(out + s * MN + e, u);
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] += u[j];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            v[j] += bias[c + j];
            if (relu) v[j] = fmaxf(v[j], 0.f);
        }
        *reinterpret_cast<uint4 *>(y + e) = bf16x8(v);
    }
}

// upconv epilogue: out [Pin][4][C] (child q = 2 i + j of input pixel (y, x)) -> y [B][2H][2W][C] + bias
__global__ void k_epi_up(const float *out, int B, int H, int W, int C, const float *bias, bf16 *y)
{
    const int n8 = B * H * W * 4 * C / 8;
    GRID_LOOP(i, n8) {
        const int e = 8 * (int)i, c = e % C, t = e / C, q = t & 3, p = t >> 2;
        const int x = p % W, yy = (p / W) % H, b = p / (W * H);
        float v[8];
        load8(out + e, v);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] += bias[c + j];
        const long long dst = (((long long)b * 2 * H + 2 * yy + q / 2) * 2 * W + 2 * x + (q & 1)) * C + c;
        *reinterpret_cast<uint4 *>(y + dst) = bf16x8(v);
    }
}

// dz = bf16(sum_splits g) * (y > 0)   (ReLU backward on the post-activation y), n = 8 n8 elements
__global__ void k_relu_back(const float *g, int splits, int n8, const bf16 *y, bf16 *dz)
{
    const long long n = 8LL * n8;
    GRID_LOOP(i, n8) {
        const int e = 8 * (int)i;
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int s = 0; s < splits; ++s) {
            float u[8];
            load8(g + s * n + e, u);
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] += u[j];
        }
        const uint4 yb = *reinterpret_cast<const uint4 *>(y + e);
        const unsigned yw[4] = {yb.x, yb.y, yb.z, yb.w};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float yv = __uint_as_float(j & 1 ? yw[j / 2] & 0xFFFF0000u : yw[j / 2] << 16);
            v[j] = yv > 0.f ? v[j] : 0.f;   // bf16 of 0 is +0, as the rounded sum masked to zero
        }
        *reinterpret_cast<uint4 *>(dz + e) = bf16x8(v);
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

// The same for many slices: 8 lanes per output sum contiguous slice ranges,
// then the lane sums are added in lane order (fixed order; out may be parts).
__global__ void k_sum_splits_wide(const float *parts, int splits, long long n, float *out)
{
    __shared__ float sh[8][32];
    const int o = threadIdx.x & 31, l = threadIdx.x >> 5;
    const long long i = blockIdx.x * 32LL + o;
    const int per = (splits + 7) / 8, s0 = l * per, s1 = min(splits, s0 + per);
    float v = 0.f;
    if (i < n)
        for (int s = s0; s < s1; ++s) v += parts[(long long)s * n + i];
    sh[l][o] = v;
    __syncthreads();
    if (l == 0 && i < n) {
        float t = sh[0][o];
        for (int j = 1; j < 8; ++j) t += sh[j][o];
        out[i] = t;
    }
}

// Column sums of x [P][C] (BF16, C a multiple of 8, C / 8 <= ET), each row r
// weighted by wrow[r] when wrow is given, over the row block [b R, (b+1) R):
// part[b][c] = sum_r wrow[r] x[r][c], and part[b][C] = sum_r wrow[r] when
// ones.  Thread t reads 16 bytes (channels 8 (t % (C/8)) ..) of rows
// t / (C/8), + ET / (C/8), ...; the row lanes are added in a fixed order.
// sum_slices then adds the blocks: a deterministic reduction over P.
constexpr int COLSUM_BLOCKS = 512;
__global__ void k_colsum_partial(const bf16 *x, const float *wrow, long long P, int C, long long R, int ones,
                                 float *part)
{
    __shared__ float sh[ET * 8];
    __shared__ float shw[ET];
    const int t = threadIdx.x, q = C / 8, per = ET / q, cg = t % q, rl = t / q;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, accw = 0.f;
    if (rl < per) {
        const long long r1 = std::min(P, (blockIdx.x + 1) * R);
        for (long long r = blockIdx.x * R + rl; r < r1; r += per) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(x + r * C) + cg);
            const float w = wrow ? wrow[r] : 1.f;
            const unsigned u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                acc[2 * j] += w * __uint_as_float(u[j] << 16);
                acc[2 * j + 1] += w * __uint_as_float(u[j] & 0xFFFF0000u);
            }
            accw += w;
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) sh[t * 8 + j] = acc[j];
    shw[t] = accw;
    __syncthreads();
    if (t < C) {   // channel t = 8 cg + j
        float v = 0.f;
        for (int l = 0; l < per; ++l) v += sh[(l * q + t / 8) * 8 + (t & 7)];
        part[(long long)blockIdx.x * (C + ones) + t] = v;
    } else if (ones && t == C) {
        float v = 0.f;
        for (int l = 0; l < per; ++l) v += shw[l * q];
        part[(long long)blockIdx.x * (C + 1) + C] = v;
    }
}

// bias gradient of an upconv from its fine-grid output gradient dy [Pfine][C]
// is the same reduction over the fine grid.

__global__ void k_maxpool(const bf16 *x, int B, int H, int W, int C, bf16 *y, unsigned char *arg)
{
    const int Ho = H / 2, Wo = W / 2, n8 = B * Ho * Wo * (C / 8);
    GRID_LOOP(i, n8) {   // 8 channels of one output pixel
        const int e = 8 * (int)i, p = e / C, c = e - p * C;
        const int xo = p % Wo, yo = (p / Wo) % Ho, b = p / (Wo * Ho);
        float best[8];
        unsigned bi[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) best[j] = -INFINITY, bi[j] = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {   // (0,0), (0,1), (1,0), (1,1): the first maximum wins
            const uint4 u = *reinterpret_cast<const uint4 *>(
                x + (((long long)b * H + 2 * yo + q / 2) * W + 2 * xo + (q & 1)) * C + c);
            const unsigned wv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float v = __uint_as_float(j & 1 ? wv[j / 2] & 0xFFFF0000u : wv[j / 2] << 16);
                if (v > best[j]) {
                    best[j] = v;
                    bi[j] = q;
                }
            }
        }
        *reinterpret_cast<uint4 *>(y + e) = bf16x8(best);
        *reinterpret_cast<uint2 *>(arg + e) = make_uint2(bi[0] | (bi[1] << 8) | (bi[2] << 16) | (bi[3] << 24),
                                                         bi[4] | (bi[5] << 8) | (bi[6] << 16) | (bi[7] << 24));
    }
}

// g_fine (FP32 accumulator, [B][H][W][C]) += scatter of dy (FP32) at the argmax
__global__ void k_maxpool_back(const float *dy, const unsigned char *arg, int B, int H, int W, int C, float *gx)
{
    const int Ho = H / 2, Wo = W / 2, n8 = B * Ho * Wo * (C / 8);
    GRID_LOOP(i, n8) {   // 8 channels of one coarse pixel; each goes to its own fine cell
        const int e = 8 * (int)i, p = e / C, c = e - p * C;
        const int xo = p % Wo, yo = (p / Wo) % Ho, b = p / (Wo * Ho);
        float d[8];
        load8(dy + e, d);
        const uint2 a = *reinterpret_cast<const uint2 *>(arg + e);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int q = (int)(((j < 4 ? a.x : a.y) >> (8 * (j & 3))) & 0xFFu);
            gx[(((long long)b * H + 2 * yo + q / 2) * W + 2 * xo + (q & 1)) * C + c + j] += d[j];
        }
    }
}

// concat [P][Ca] ++ [P][Cb] -> [P][Ca+Cb]  (8-channel chunks)
__global__ void k_concat(const bf16 *a, int Ca, const bf16 *b, int Cb, int P, bf16 *y)
{
    const int C = Ca + Cb, n8 = P * (C / 8);
    GRID_LOOP(i, n8) {
        const int e = 8 * (int)i, p = e / C, c = e - p * C;
        *reinterpret_cast<uint4 *>(y + e) = c < Ca ? *reinterpret_cast<const uint4 *>(a + (long long)p * Ca + c)
                                                   : *reinterpret_cast<const uint4 *>(b + (long long)p * Cb + c - Ca);
    }
}

// split the FP32 gradient of a concat: first Ca channels -> ga (bf16), the rest added to gb (FP32)
__global__ void k_concat_back(const float *g, int Ca, int Cb, int P, bf16 *ga, float *gb)
{
    const int C = Ca + Cb, n8 = P * (C / 8);
    GRID_LOOP(i, n8) {
        const int e = 8 * (int)i, p = e / C, c = e - p * C;
        float v[8];
        load8(g + e, v);
        if (c < Ca) {
            *reinterpret_cast<uint4 *>(ga + (long long)p * Ca + c) = bf16x8(v);
        } else {
            float *d = gb + (long long)p * Cb + c - Ca;
            float u[8];
            load8(d, u);
            *reinterpret_cast<float4 *>(d) = make_float4(u[0] + v[0], u[1] + v[1], u[2] + v[2], u[3] + v[3]);
            *reinterpret_cast<float4 *>(d + 4) = make_float4(u[4] + v[4], u[5] + v[5], u[6] + v[6], u[7] + v[7]);
        }
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

// upconv weights w [Cin][4 Cout] -> wt [4 Cout][Cin]
__global__ void k_transpose_up(const bf16 *w, int Cin, int N4, bf16 *wt)
{
    GRID_LOOP(i, (long long)Cin * N4) {
        const int n = (int)(i % N4), ci = (int)(i / N4);
        wt[(long long)n * Cin + ci] = w[i];
    }
}

// input [B][2][H][W] FP32 (NCHW) -> [B][H][W][2] BF16
__global__ void k_pack_input(const float *x, int B, int H, int W, bf16 *y)
{
    const long long hw = (long long)H * W, n = B * hw;
    GRID_LOOP(p, n) {   // pixel p: channels 0, 1 from the two input planes, 2 .. XIN_C - 1 zero
        const long long b = p / hw, r = p - b * hw;
        const unsigned c0 = __bfloat16_as_ushort(__float2bfloat16_rn(x[(b * 2) * hw + r]));
        const unsigned c1 = __bfloat16_as_ushort(__float2bfloat16_rn(x[(b * 2 + 1) * hw + r]));
        uint4 *d = reinterpret_cast<uint4 *>(y + p * XIN_C);
        d[0] = make_uint4(c0 | (c1 << 16), 0, 0, 0);
        d[1] = make_uint4(0, 0, 0, 0);
    }
}

// first-layer weights w [Cout][9][2] -> wp [Cout][9][XIN_C] (zero beyond channel 1)
__global__ void k_pad_w0(const bf16 *w, int Cout, bf16 *wp)
{
    GRID_LOOP(i, (long long)Cout * 9 * XIN_C) {
        const int c = (int)(i % XIN_C);
        wp[i] = c < 2 ? w[(i / XIN_C) * 2 + c] : __float2bfloat16_rn(0.f);
    }
}

// first-layer weight gradient: g [Cout][9][2] <- gp [Cout][9][XIN_C], channels 0, 1
__global__ void k_unpad_w0(const float *gp, int Cout, float *g)
{
    GRID_LOOP(i, (long long)Cout * 9 * 2) g[i] = gp[(i / 2) * XIN_C + (i % 2)];
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
    __shared__ double sh[ET];
    double a = 0.0;
    for (int i = threadIdx.x; i < nb; i += ET) a += part[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = ET / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = 0.5 * sh[0] / (double)P;
}

// head backward: gx[p][c] = dout[p] w[c] (FP32); dw[c] = sum_p dout[p] x[p][c] and db = sum dout by
// k_colsum_partial (rows weighted by dout, a ones column)
__global__ void k_head_back_x(const float *dout, int P, int C, const bf16 *w, float *gx)
{
    const int n8 = P * (C / 8);
    GRID_LOOP(i, n8) {
        const int e = 8 * (int)i, p = e / C, c = e - p * C;
        const float d = dout[p];
        float4 lo, hi;
        lo.x = d * __bfloat162float(w[c]), lo.y = d * __bfloat162float(w[c + 1]);
        lo.z = d * __bfloat162float(w[c + 2]), lo.w = d * __bfloat162float(w[c + 3]);
        hi.x = d * __bfloat162float(w[c + 4]), hi.y = d * __bfloat162float(w[c + 5]);
        hi.z = d * __bfloat162float(w[c + 6]), hi.w = d * __bfloat162float(w[c + 7]);
        *reinterpret_cast<float4 *>(gx + e) = lo;
        *reinterpret_cast<float4 *>(gx + e + 4) = hi;
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
    float *bpart = nullptr;   // column-sum block partials [COLSUM_BLOCKS][8 C + 1]
    bf16 *w0p = nullptr;      // first-layer weights padded to XIN_C input channels
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
// (w, cin: the first layer's padded weights and input channels; NULL / 0: the layer's own)
void conv_fwd(aafwi_unet *u, const Conv &c, const bf16 *x, int B, int H, int W, bf16 *y, cudaStream_t st,
              const bf16 *w = nullptr, int cin = 0)
{
    const int s = unet_conv3_fwd(x, w ? w : wb(u, c), B, H, W, cin ? cin : c.Cin, c.Cout, u->P + c.b, y, u->gemm,
                                 u->gemm_size, st);
    if (s > 0) {   // split slices: sum, bias, ReLU, BF16
        const long long MN = (long long)B * H * W * c.Cout;
        count_launch();
        k_epi<<<nblk(MN / 8), ET, 0, st>>>(u->gemm, s, (int)(MN / 8), c.Cout, u->P + c.b, 1, y);
    }
}

void up_fwd(aafwi_unet *u, const Conv &c, const bf16 *x, int B, int H, int W, bf16 *y, cudaStream_t st)
{
    count_launch();
    k_transpose_up<<<nblk(c.nw()), ET, 0, st>>>(wb(u, c), c.Cin, 4 * c.Cout, u->Wt);
    unet_up_fwd(x, u->Wt, B, H, W, c.Cin, c.Cout, u->gemm, st);
    count_launch();
    k_epi_up<<<nblk((long long)B * H * W * c.Cout / 2), ET, 0, st>>>(u->gemm, B, H, W, c.Cout, u->P + c.b, y);
}

// out[i] = sum over the split slices of parts [splits][n] (out may be parts)
void sum_slices(const float *parts, int splits, long long n, float *out, cudaStream_t st)
{
    count_launch();
    if (splits <= 8) k_sum_splits<<<nblk(n), ET, 0, st>>>(parts, splits, n, out);
    else k_sum_splits_wide<<<(unsigned)((n + 31) / 32), ET, 0, st>>>(parts, splits, n, out);
}

// out[c] = sum_r wrow[r] x[r][c] over the P rows of x [P][C] (wrow NULL: 1),
// and out[C] = sum_r wrow[r] when ones
void colsum(aafwi_unet *u, const bf16 *x, const float *wrow, long long P, int C, int ones, float *out, cudaStream_t st)
{
    const long long nb = std::max(1LL, std::min<long long>(COLSUM_BLOCKS, P / 512));
    const long long R = (P + nb - 1) / nb;
    count_launch();
    k_colsum_partial<<<(unsigned)nb, ET, 0, st>>>(x, wrow, P, C, R, ones, u->bpart);
    sum_slices(u->bpart, (int)nb, C + ones, out, st);
}

// db = sum over the P rows of dz [P][C]
void bias_grad(aafwi_unet *u, const bf16 *dz, long long P, int C, float *db, cudaStream_t st)
{
    colsum(u, dz, nullptr, P, C, 0, db, st);
}

// K splits a weight gradient may write into u->gemm
int wgrad_cap(const aafwi_unet *u, const Conv &c) { return (int)std::max(1LL, std::min(1024LL, u->gemm_size / c.nw())); }

// Backward of y = relu(conv3(x) + b): gy (FP32 [P][Cout]) -> dW, db (into u->G),
// returns gx in FP32 (u->gemm, its split slices summed into the first) when want_gx.
// xc: channels of x as stored (the first layer's padded input), 0: c.Cin
void conv_back(aafwi_unet *u, const Conv &c, const bf16 *x, const bf16 *y, const float *gy, int B, int H, int W,
               bool want_gx, cudaStream_t st, int xc = 0)
{
    const long long P = (long long)B * H * W;
    count_launch();
    k_relu_back<<<nblk(P * c.Cout / 8), ET, 0, st>>>(gy, 1, (int)(P * c.Cout / 8), y, u->gb1);
    bias_grad(u, u->gb1, P, c.Cout, u->G + c.b, st);
    if (xc && xc != c.Cin) {   // weight gradient at xc input channels, then the first c.Cin of them
        const long long nwp = 9LL * xc * c.Cout;
        const int cap = (int)std::max(1LL, std::min(1024LL, u->gemm_size / nwp));
        const int s = unet_conv3_wgrad(u->gb1, x, B, H, W, xc, c.Cout, cap, u->gemm, st);
        sum_slices(u->gemm, s, nwp, u->bpart, st);
        count_launch();
        k_unpad_w0<<<nblk(c.nw()), ET, 0, st>>>(u->bpart, c.Cout, u->G + c.w);
    } else {
        const int s = unet_conv3_wgrad(u->gb1, x, B, H, W, c.Cin, c.Cout, wgrad_cap(u, c), u->gemm, st);
        sum_slices(u->gemm, s, c.nw(), u->G + c.w, st);
    }
    if (want_gx) {
        count_launch();
        bf16 *wt = u->Wt;
        k_transpose_w<<<nblk(c.nw()), ET, 0, st>>>(wb(u, c), c.Cout, c.Cin, wt);
        const int sx = unet_conv3_dgrad(u->gb1, wt, B, H, W, c.Cin, c.Cout, u->gemm, u->gemm_size, st);
        if (sx > 1) sum_slices(u->gemm, sx, P * c.Cin, u->gemm, st);   // the slices, in place into the first
    }
}

// Backward of y = upconv(x) + b (no activation): gy (BF16 [B][2H][2W][Cout])
void up_back(aafwi_unet *u, const Conv &c, const bf16 *x, const bf16 *gy, int B, int H, int W, cudaStream_t st)
{
    const long long Pin = (long long)B * H * W;
    bias_grad(u, gy, 4 * Pin, c.Cout, u->G + c.b, st);
    const int s = unet_up_wgrad(x, gy, B, H, W, c.Cin, c.Cout, wgrad_cap(u, c), u->gemm, st);
    sum_slices(u->gemm, s, c.nw(), u->G + c.w, st);
    unet_up_dgrad(gy, wb(u, c), B, H, W, c.Cin, c.Cout, u->gemm, st);
}

void forward(aafwi_unet *u, const float *xin, int B, cudaStream_t st)
{
    count_launch();
    k_pack_input<<<nblk((long long)B * u->H * u->W), ET, 0, st>>>(xin, B, u->H, u->W, u->xin);
    count_launch();
    k_pad_w0<<<nblk(9LL * XIN_C * u->C), ET, 0, st>>>(wb(u, u->L[0]), u->C, u->w0p);
    const bf16 *x = u->xin;
    int li = 0;
    for (int l = 0; l < 3; ++l) {
        const int H = Hl(u, l), W = Wl(u, l);
        if (l == 0) conv_fwd(u, u->L[li++], x, B, H, W, u->ea[l], st, u->w0p, XIN_C);
        else conv_fwd(u, u->L[li++], x, B, H, W, u->ea[l], st);
        conv_fwd(u, u->L[li++], u->ea[l], B, H, W, u->eb[l], st);
        count_launch();
        k_maxpool<<<nblk((long long)B * H / 2 * W / 2 * Cl(u, l) / 8), ET, 0, st>>>(u->eb[l], B, H, W, Cl(u, l), u->pool[l], u->arg[l]);
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
        k_concat<<<nblk(P * 2 * Cl(u, l) / 8), ET, 0, st>>>(u->up[l], Cl(u, l), u->eb[l], Cl(u, l), (int)P, u->cat[l]);
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
    colsum(u, u->db[0], u->dout, P0, C, 1, u->G + u->head_w, st);   // head weights, then its bias (head_b = head_w + C)
    count_launch();
    k_head_back_x<<<nblk(P0 * C / 8), ET, 0, st>>>(u->dout, (int)P0, C, u->Pb + u->head_w, u->gacc);
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
        k_concat_back<<<nblk(P * 2 * Cv / 8), ET, 0, st>>>(u->gemm, Cv, Cv, (int)P, u->gb2, gskip[l]);
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
        k_maxpool_back<<<nblk((long long)B * H / 2 * W / 2 * Cv / 8), ET, 0, st>>>(u->gemm, u->arg[l], B, H, W, Cv,
                                                                                gskip[l]);
        conv_back(u, u->L[li--], u->ea[l], u->eb[l], gskip[l], B, H, W, true, st);          // enc b
        const bf16 *xin = l == 0 ? u->xin : u->pool[l - 1];
        conv_back(u, u->L[li--], xin, u->ea[l], u->gemm, B, H, W, l > 0, st, l == 0 ? XIN_C : 0);   // enc a
    }
}

void loss_and_grad(aafwi_unet *u, const float *xin, const float *target, int B, cudaStream_t st)
{
    forward(u, xin, B, st);
    const long long P = (long long)B * u->H * u->W;
    const int nb = (int)std::min<long long>(4096, (P + ET - 1) / ET);
    count_launch(2);
    k_mse<<<nb, ET, 0, st>>>(u->out, target, P, u->dout, u->lpart);
    k_mse_finish<<<1, ET, 0, st>>>(u->lpart, nb, P, u->loss);
    backward(u, B, st);
}

}  // namespace

extern "C" {

int aafwi_unet_create(int Bmax, int H, int W, int C, aafwi_unet **out)
{
    if (!out || Bmax < 1 || H < 8 || W < 8 || H % 8 || W % 8 || C < 8 || C % 8 || C > 1024 ||
        (long long)Bmax * H * W * 16 * C >= INT_MAX)
        return uerr(nullptr, AAFWI_ERR_ARG,
                    "unet_create: need Bmax >= 1, H, W multiples of 8, C multiple of 8 (at most 1024), "
                    "Bmax H W 16 C below 2^31");
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
    // largest GEMM output (the split slices of the weight gradients are bounded by this size)
    long long gs = 0;
    for (int l = 0; l < 4; ++l) {
        const long long P = P0 >> (2 * l);
        gs = std::max(gs, P * (8LL * C) * 2);        // activations x widest channels (concat)
    }
    u->gemm_size = gs;
    bool ok = ualloc(u, &u->P, off) && ualloc(u, &u->G, off) && ualloc(u, &u->Mm, off) && ualloc(u, &u->Vv, off) &&
              ualloc(u, &u->Pb, off) && ualloc(u, &u->Wt, maxw) && ualloc(u, &u->xin, P0 * XIN_C) && ualloc(u, &u->w0p, 9LL * XIN_C * C) &&
              ualloc(u, &u->gemm, gs) && ualloc(u, &u->gacc, P0 * 8 * C) && ualloc(u, &u->gacc2, P0 * 2 * C) &&
              ualloc(u, &u->gb1, P0 * 8 * C) && ualloc(u, &u->gb2, P0 * 8 * C) && ualloc(u, &u->out, P0) &&
              ualloc(u, &u->dout, P0) && ualloc(u, &u->lpart, 4096) && ualloc(u, &u->loss, 1) &&
              ualloc(u, &u->bpart, (size_t)COLSUM_BLOCKS * (8 * C + 1));
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
        s = unet_conv3_fwd(x, y, B, H, W, Cin, Cout, nullptr, nullptr, out, cap, st);
    } else if (op == AAFWI_CONV3_DGRAD) {
        const long long cap = splits > 0 ? std::min(out_cap, splits * MN) : out_cap;
        s = unet_conv3_dgrad(x, y, B, H, W, Cin, Cout, out, cap, st);
    } else {
        const long long cap = std::min(1024LL, out_cap / MN);
        s = unet_conv3_wgrad(x, y, B, H, W, Cin, Cout, (int)(splits > 0 ? std::min<long long>(splits, cap) : cap), out,
                             st);
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
