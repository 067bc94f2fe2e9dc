// unet_kernels.cu -- BF16 tensor-core kernels of the learned preconditioner
// (a small U-Net mapping [gradient, model] to a model update; not part of the
// paper, which has no learned component).
//
// Every convolution-like operation is an implicit GEMM  C[M][N] = sum_k
// A(m, k) B(k, n)  on BF16 operands with FP32 accumulation, computed with
// mma.sync.m16n8k16 tensor-core instructions.  Activations are NHWC BF16.
//   conv3x3 forward   M = pixels, N = Cout, K = 9 Cin   A = im2col(x), B = w[Cout][9][Cin]
//   conv3x3 dgrad     M = pixels, N = Cin,  K = 9 Cout  A = im2col(dz) flipped, B = wt[Cin][9][Cout]
//   conv3x3 wgrad     M = Cout,   N = 9 Cin, K = pixels A = dz^T, B = im2col(x)   (split over pixels)
//   upconv2x2 forward M = pixels_in, N = 4 Cout, K = Cin      (output scattered to the 2x2 children)
//   upconv2x2 dgrad   M = pixels_in, N = Cin,    K = 4 Cout   (gathers the 2x2 children)
//   upconv2x2 wgrad   M = Cin,       N = 4 Cout, K = pixels_in
// CTA tile 64 x 64 x 32, 4 warps each owning 32 x 32 (2 x 4 mma tiles);
// operands are staged K-contiguous in shared memory and fed to the
// fragments with 32-bit loads.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace aafwi {
namespace unet {

constexpr int BM = 64, BN = 64, BK = 32, KP = BK + 8;   // KP: padded row (bank spread)

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Operand gathers, one per GEMM mode.  fillA / fillB write 16 consecutive K
// elements of one row of the A (M x K) or B^T (N x K) tile as raw BF16 bits,
// 0 outside the tensor, the zero padding or the K range.
struct ConvGeom {
    int B, H, W;       // batch and spatial size of the GEMM's pixel grid
    int Cin, Cout;
};

enum Mode { CONV_FWD = 0, CONV_DGRAD = 1, CONV_WGRAD = 2, UP_FWD = 3, UP_DGRAD = 4, UP_WGRAD = 5 };

template <int MODE>
struct Op {
    const unsigned short *a, *b;  // operand tensors as raw BF16 bits
    ConvGeom g;
    int M, N, K;
    int klen;                     // K extent of one split (multiple of BK)
};

struct Pix {
    int b, y, x;
};

__device__ __forceinline__ Pix pix(const ConvGeom &g, int p)
{
    const int hw = g.H * g.W;
    Pix q;
    q.b = p / hw;
    const int r = p - q.b * hw;
    q.y = r / g.W;
    q.x = r - q.y * g.W;
    return q;
}

// im2col segment: element k = tap * C + c of pixel q, tap offsets (sign * (ky-1, kx-1))
__device__ __forceinline__ void im2col16(const unsigned short *t, const ConvGeom &g, int C, Pix q, int k0, int ke,
                                         int sign, unsigned short *dst)
{
    int tap = k0 / C, c = k0 - tap * C;
    for (int i = 0; i < 16; ++i) {
        const int k = k0 + i;
        unsigned short v = 0;
        if (k < ke) {
            const int yy = q.y + sign * (tap / 3 - 1), xx = q.x + sign * (tap % 3 - 1);
            if (yy >= 0 && yy < g.H && xx >= 0 && xx < g.W)
                v = t[(((long long)q.b * g.H + yy) * g.W + xx) * C + c];
        }
        dst[i] = v;
        if (++c == C) {
            c = 0;
            ++tap;
        }
    }
}

template <int MODE>
__device__ __forceinline__ void fillA(const Op<MODE> &o, int m, int k0, int ke, unsigned short *dst)
{
    const ConvGeom &g = o.g;
    if (MODE == CONV_FWD || MODE == CONV_DGRAD) {
        // m = pixel; x or dz in NHWC [B][H][W][C]
        im2col16(o.a, g, MODE == CONV_FWD ? g.Cin : g.Cout, pix(g, m), k0, ke, MODE == CONV_FWD ? 1 : -1, dst);
    } else if (MODE == CONV_WGRAD || MODE == UP_WGRAD) {
        // m = channel, k = pixel: t [P][C]
        const int C = MODE == CONV_WGRAD ? g.Cout : g.Cin;
        for (int i = 0; i < 16; ++i) dst[i] = k0 + i < ke ? o.a[(long long)(k0 + i) * C + m] : 0;
    } else if (MODE == UP_FWD) {
        // m = input pixel, k = cin: x [Pin][Cin]
        for (int i = 0; i < 16; ++i) dst[i] = k0 + i < ke ? o.a[(long long)m * g.Cin + k0 + i] : 0;
    } else {  // UP_DGRAD: m = coarse pixel, k = q * Cout + co; dy [B][2H][2W][Cout]
        const Pix q0 = pix(g, m);
        int q = k0 / g.Cout, co = k0 - q * g.Cout;
        for (int i = 0; i < 16; ++i) {
            unsigned short v = 0;
            if (k0 + i < ke) {
                const int Y = 2 * q0.y + q / 2, X = 2 * q0.x + (q & 1);
                v = o.a[(((long long)q0.b * 2 * g.H + Y) * 2 * g.W + X) * g.Cout + co];
            }
            dst[i] = v;
            if (++co == g.Cout) {
                co = 0;
                ++q;
            }
        }
    }
}

template <int MODE>
__device__ __forceinline__ void fillB(const Op<MODE> &o, int n, int k0, int ke, unsigned short *dst)
{
    const ConvGeom &g = o.g;
    if (MODE == CONV_FWD || MODE == CONV_DGRAD || MODE == UP_DGRAD) {
        // weights stored N-major with K contiguous: w[n][k]
        for (int i = 0; i < 16; ++i) dst[i] = k0 + i < ke ? o.b[(long long)n * o.K + k0 + i] : 0;
    } else if (MODE == UP_FWD) {  // w [Cin][4 Cout]: B(k = cin, n)
        for (int i = 0; i < 16; ++i) dst[i] = k0 + i < ke ? o.b[(long long)(k0 + i) * o.N + n] : 0;
    } else if (MODE == CONV_WGRAD) {  // n = tap * Cin + cin, k = pixel: x [B][H][W][Cin]
        const int tap = n / g.Cin, c = n - tap * g.Cin;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        for (int i = 0; i < 16; ++i) {
            unsigned short v = 0;
            if (k0 + i < ke) {
                const Pix q = pix(g, k0 + i);
                const int yy = q.y + dy, xx = q.x + dx;
                if (yy >= 0 && yy < g.H && xx >= 0 && xx < g.W)
                    v = o.b[(((long long)q.b * g.H + yy) * g.W + xx) * g.Cin + c];
            }
            dst[i] = v;
        }
    } else {  // UP_WGRAD: n = q * Cout + co, k = coarse pixel: dy [B][2H][2W][Cout]
        const int q = n / g.Cout, co = n - q * g.Cout;
        for (int i = 0; i < 16; ++i) {
            unsigned short v = 0;
            if (k0 + i < ke) {
                const Pix p = pix(g, k0 + i);
                const int Y = 2 * p.y + q / 2, X = 2 * p.x + (q & 1);
                v = o.b[(((long long)p.b * 2 * g.H + Y) * 2 * g.W + X) * g.Cout + co];
            }
            dst[i] = v;
        }
    }
}

// One CTA: a BM x BN tile of C over its K split [kb, kb + klen).  The FP32
// result goes to out[(split * M + m) * N + n] (split = blockIdx.z).
template <int MODE>
__global__ void __launch_bounds__(128) k_gemm(const Op<MODE> o, float *out)
{
    __shared__ __align__(16) unsigned short As[BM][KP];
    __shared__ __align__(16) unsigned short Bs[BN][KP];
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kb = blockIdx.z * o.klen;
    const int ke = min(kb + o.klen, o.K);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int grp = lane >> 2, tig = lane & 3;
    const int fr = tid >> 1, fk = (tid & 1) * 16;     // staging: row fr, 16 K from fk
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    for (int k0 = kb; k0 < ke; k0 += BK) {
        unsigned short seg[16];
        if (m0 + fr < o.M) fillA<MODE>(o, m0 + fr, k0 + fk, ke, seg);
        else
            for (int i = 0; i < 16; ++i) seg[i] = 0;
        for (int i = 0; i < 16; i += 2)
            *reinterpret_cast<uint32_t *>(&As[fr][fk + i]) = seg[i] | ((uint32_t)seg[i + 1] << 16);
        if (n0 + fr < o.N) fillB<MODE>(o, n0 + fr, k0 + fk, ke, seg);
        else
            for (int i = 0; i < 16; ++i) seg[i] = 0;
        for (int i = 0; i < 16; i += 2)
            *reinterpret_cast<uint32_t *>(&Bs[fr][fk + i]) = seg[i] | ((uint32_t)seg[i + 1] << 16);
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + 16 * i + grp;
                af[i][0] = *reinterpret_cast<const uint32_t *>(&As[r][ks + 2 * tig]);
                af[i][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + 2 * tig]);
                af[i][2] = *reinterpret_cast<const uint32_t *>(&As[r][ks + 8 + 2 * tig]);
                af[i][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + 8 + 2 * tig]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + 8 * j + grp;
                bf[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[c][ks + 2 * tig]);
                bf[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[c][ks + 8 + 2 * tig]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
        }
        __syncthreads();
    }
    float *dst = out + (long long)blockIdx.z * o.M * o.N;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = m0 + wm + 16 * i + grp, c = n0 + wn + 8 * j + 2 * tig;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int rr = r + (e >> 1) * 8, cc = c + (e & 1);
                if (rr < o.M && cc < o.N) dst[(long long)rr * o.N + cc] = acc[i][j][e];
            }
        }
}

template <int MODE>
int gemm(const __nv_bfloat16 *a, const __nv_bfloat16 *b, ConvGeom g, int M, int N, int K, int splits,
         float *out, cudaStream_t st)
{
    Op<MODE> o{reinterpret_cast<const unsigned short *>(a), reinterpret_cast<const unsigned short *>(b), g,
               M, N, K, 0};
    const int kchunks = (K + BK - 1) / BK;
    splits = max(1, min(splits, kchunks));
    o.klen = ((kchunks + splits - 1) / splits) * BK;
    splits = (K + o.klen - 1) / o.klen;
    dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN, splits);
    count_launch();
    k_gemm<MODE><<<grid, 128, 0, st>>>(o, out);
    return splits;
}

}  // namespace unet

using namespace unet;

// ---------------------------------------------------------------------------
// launchers used by the U-Net runtime (unet.cu)
// ---------------------------------------------------------------------------

// FP32 GEMM results for one operation, [splits][M][N]; `splits` > 1 only for
// the weight gradients (K = pixels); each returns the number of splits used.
int unet_conv3_fwd(const __nv_bfloat16 *x, const __nv_bfloat16 *w, int B, int H, int W, int Cin, int Cout,
                    float *out, cudaStream_t st)
{
    ConvGeom g{B, H, W, Cin, Cout};
    return gemm<CONV_FWD>(x, w, g, B * H * W, Cout, 9 * Cin, 1, out, st);
}

int unet_conv3_dgrad(const __nv_bfloat16 *dz, const __nv_bfloat16 *wt, int B, int H, int W, int Cin, int Cout,
                      float *out, cudaStream_t st)
{
    ConvGeom g{B, H, W, Cin, Cout};
    return gemm<CONV_DGRAD>(dz, wt, g, B * H * W, Cin, 9 * Cout, 1, out, st);
}

int unet_conv3_wgrad(const __nv_bfloat16 *dz, const __nv_bfloat16 *x, int B, int H, int W, int Cin, int Cout,
                      int splits, float *out, cudaStream_t st)
{
    ConvGeom g{B, H, W, Cin, Cout};
    return gemm<CONV_WGRAD>(dz, x, g, Cout, 9 * Cin, B * H * W, splits, out, st);
}

int unet_up_fwd(const __nv_bfloat16 *x, const __nv_bfloat16 *w, int B, int H, int W, int Cin, int Cout,
                 float *out, cudaStream_t st)
{
    ConvGeom g{B, H, W, Cin, Cout};
    return gemm<UP_FWD>(x, w, g, B * H * W, 4 * Cout, Cin, 1, out, st);
}

int unet_up_dgrad(const __nv_bfloat16 *dy, const __nv_bfloat16 *w, int B, int H, int W, int Cin, int Cout,
                   float *out, cudaStream_t st)
{
    ConvGeom g{B, H, W, Cin, Cout};
    return gemm<UP_DGRAD>(dy, w, g, B * H * W, Cin, 4 * Cout, 1, out, st);
}

int unet_up_wgrad(const __nv_bfloat16 *x, const __nv_bfloat16 *dy, int B, int H, int W, int Cin, int Cout,
                   int splits, float *out, cudaStream_t st)
{
    ConvGeom g{B, H, W, Cin, Cout};
    return gemm<UP_WGRAD>(x, dy, g, Cin, 4 * Cout, B * H * W, splits, out, st);
}

}  // namespace aafwi
