// unet_kernels.cu -- BF16 tensor-core kernels of the learned preconditioner
// (a small U-Net mapping [gradient, model] to a model update; not part of the
// paper, which has no learned component).
//
// Every convolution-like operation is an implicit GEMM  C[M][N] = sum_k
// A(m, k) B(k, n)  on BF16 operands with FP32 accumulation, computed with
// tcgen05.mma (accumulator in tensor memory).  Activations are NHWC BF16.
//   conv3x3 forward   M = pixels, N = Cout, K = 9 Cin   A = im2col(x), B = w[Cout][9][Cin]
//   conv3x3 dgrad     M = pixels, N = Cin,  K = 9 Cout  A = im2col(dz) flipped, B = wt[Cin][9][Cout]
//   conv3x3 wgrad     M = Cout,   N = 9 Cin, K = pixels A = dz^T, B = im2col(x)   (split over pixels)
//   upconv2x2 forward M = pixels_in, N = 4 Cout, K = Cin      (output scattered to the 2x2 children)
//   upconv2x2 dgrad   M = pixels_in, N = Cin,    K = 4 Cout   (gathers the 2x2 children)
//   upconv2x2 wgrad   M = Cin,       N = 4 Cout, K = pixels_in
// Two forms:
//   * k_conv_win / k_wgrad_win: the 3x3 layers whose channels are 16 times a
//     power of two, as windowed GEMMs -- the padded input is staged once per
//     CTA and every tap reads it at a row offset (no im2col); see k_conv_win;
//   * k_gemm_tc: the upconvs and any 3x3 layer with other channel counts, with
//     the operands gathered per K chunk of 32 (CTA tile 128 x 64).
#include <cuda_bf16.h>

#include "internal.cuh"

namespace aafwi {
namespace unet {

constexpr int BK = 32;   // K granularity of the splits

// Operand gathers of the K-major modes (forward and data gradients).  fillA /
// fillB write 16 consecutive K elements of one row of the A (M x K) or B^T
// (N x K) tile as raw BF16 bits, 0 outside the tensor, the zero padding or the
// K range.  The weight gradients gather MN-major (wgrad_a8 / wgrad_b8).
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

// 16 consecutive BF16 values, as two 16-byte loads from a 32-byte aligned
// address (element by element otherwise).
__device__ __forceinline__ void load16(const unsigned short *p, unsigned short *dst)
{
    if (reinterpret_cast<uintptr_t>(p) & 31) {
#pragma unroll
        for (int i = 0; i < 16; ++i) dst[i] = p[i];
        return;
    }
    const uint4 lo = __ldg(reinterpret_cast<const uint4 *>(p)), hi = __ldg(reinterpret_cast<const uint4 *>(p) + 1);
    const unsigned w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        dst[2 * i] = (unsigned short)(w[i] & 0xFFFFu);
        dst[2 * i + 1] = (unsigned short)(w[i] >> 16);
    }
}

// im2col segment: element k = tap * C + c of pixel q, tap offsets (sign * (ky-1, kx-1))
__device__ __forceinline__ void im2col16(const unsigned short *t, const ConvGeom &g, int C, Pix q, int k0, int ke,
                                         int sign, unsigned short *dst)
{
    int tap = k0 / C, c = k0 - tap * C;
    if ((C & 15) == 0 && k0 + 16 <= ke) {   // one tap, 16 consecutive channels (k0 is a multiple of 16)
        const int yy = q.y + sign * (tap / 3 - 1), xx = q.x + sign * (tap % 3 - 1);
        if (yy >= 0 && yy < g.H && xx >= 0 && xx < g.W) {
            load16(t + (((long long)q.b * g.H + yy) * g.W + xx) * C + c, dst);
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) dst[i] = 0;
        }
        return;
    }
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
    } else if (MODE == UP_FWD) {
        // m = input pixel, k = cin: x [Pin][Cin]
        if ((g.Cin & 15) == 0 && k0 + 16 <= ke) load16(o.a + (long long)m * g.Cin + k0, dst);
        else
            for (int i = 0; i < 16; ++i) dst[i] = k0 + i < ke ? o.a[(long long)m * g.Cin + k0 + i] : 0;
    } else {  // UP_DGRAD: m = coarse pixel, k = q * Cout + co; dy [B][2H][2W][Cout]
        const Pix q0 = pix(g, m);
        int q = k0 / g.Cout, co = k0 - q * g.Cout;
        if ((g.Cout & 15) == 0 && k0 + 16 <= ke) {   // 16 channels of one child pixel
            const int Y = 2 * q0.y + q / 2, X = 2 * q0.x + (q & 1);
            load16(o.a + (((long long)q0.b * 2 * g.H + Y) * 2 * g.W + X) * g.Cout + co, dst);
            return;
        }
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
    if (MODE == CONV_FWD || MODE == CONV_DGRAD || MODE == UP_DGRAD || MODE == UP_FWD) {
        // weights stored N-major with K contiguous: w[n][k] (the upconv forward takes w^T [4 Cout][Cin])
        if ((o.K & 15) == 0 && k0 + 16 <= ke) load16(o.b + (long long)n * o.K + k0, dst);
        else
            for (int i = 0; i < 16; ++i) dst[i] = k0 + i < ke ? o.b[(long long)n * o.K + k0 + i] : 0;
    }
}

// ---------------------------------------------------------------------------
// 5th-generation tensor cores (tcgen05): the same implicit GEMMs with the
// accumulator in tensor memory.  CTA tile TM x TN, K in chunks of TK: the 128
// threads gather the chunk's A (TM x TK) and B (TN x TK) operands into shared
// memory in the K-major, unswizzled operand layout (8 x 8 BF16 core matrices,
// 8 rows x 16 bytes); one thread issues TK/16 MMAs (128 x 64 x 16 each) and
// commits them to an mbarrier, which every thread waits for (bounded) before
// the next chunk overwrites the operands.  The epilogue reads the FP32
// accumulator from tensor memory (warp w: lanes 32w .. 32w+31 = tile rows).
// ---------------------------------------------------------------------------

constexpr int TM = 128, TN = 64, TK = 32;
static_assert(TK == BK, "K splits are laid out in multiples of BK");

// Error word of the U-Net kernels (bit 0: a tensor-core commit wait ran out).
__device__ int g_unet_err;
int *unet_error_word()
{
    static int *p = nullptr;
    if (!p) cudaGetSymbolAddress((void **)&p, g_unet_err);
    return p;
}

}  // namespace unet

// Host: the U-Net error word (then cleared); call after the work has been synchronised.
int unet_take_error()
{
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, unet::g_unet_err, sizeof(int)) != cudaSuccess) return -1;
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbol(unet::g_unet_err, &z, sizeof(int));
    }
    return v;
}

namespace unet {
constexpr int T_LBO = 128;                  // bytes between core matrices adjacent along K
constexpr int T_SBO = TK / 8 * 128;         // bytes between 8-row groups
constexpr long long T_WAIT_LIMIT = 1LL << 22;

__device__ __forceinline__ unsigned tc_off(int r, int k)
{
    return (unsigned)((r >> 3) * T_SBO + (k >> 3) * T_LBO + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ unsigned tc_smem(const void *p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (8-row group) byte offsets, descriptor version 1, no swizzle.  Every field
// is in 16-byte units (14 bits: addresses and offsets below 256 KB).
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr, unsigned lbo, unsigned sbo)
{
    return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFF) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr) { return tc_desc(addr, T_LBO, T_SBO); }

// Instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, N = TN, M = TM.
constexpr unsigned TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(TN >> 3) << 17) |
                              ((unsigned)(TM >> 4) << 24);
// The same with A and B MN-major (bits 15, 16).
constexpr unsigned TC_IDESC_MN = TC_IDESC | (1u << 15) | (1u << 16);

__device__ __forceinline__ bool tc_wait(unsigned bar, unsigned parity)
{
    for (long long i = 0; i < T_WAIT_LIMIT; ++i) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_store16(unsigned char *tile, int r, int k, const unsigned short (&seg)[16])
{
    uint4 lo, hi;
    lo.x = seg[0] | ((unsigned)seg[1] << 16); lo.y = seg[2] | ((unsigned)seg[3] << 16);
    lo.z = seg[4] | ((unsigned)seg[5] << 16); lo.w = seg[6] | ((unsigned)seg[7] << 16);
    hi.x = seg[8] | ((unsigned)seg[9] << 16); hi.y = seg[10] | ((unsigned)seg[11] << 16);
    hi.z = seg[12] | ((unsigned)seg[13] << 16); hi.w = seg[14] | ((unsigned)seg[15] << 16);
    *reinterpret_cast<uint4 *>(tile + tc_off(r, k)) = lo;
    *reinterpret_cast<uint4 *>(tile + tc_off(r, k + 8)) = hi;
}

// Weight gradients (K = pixels) keep their operands MN-major: in NHWC the
// channels of one pixel are contiguous, so a chunk's A (M = channels) and B
// (N = tap x channel or child x channel) are gathered as 8-element (16-byte)
// runs along M / N for each of the chunk's TK pixels.  MN-major core matrix:
// 8 K-rows x 16 bytes (8 MN elements); same LBO (K groups) / SBO (MN groups).
__device__ __forceinline__ unsigned tc_off_mn(int mn, int k)
{
    return (unsigned)((mn >> 3) * T_SBO + (k >> 3) * T_LBO + (k & 7) * 16 + (mn & 7) * 2);
}

__device__ __forceinline__ uint4 ld8(const unsigned short *p)
{
    if (reinterpret_cast<uintptr_t>(p) & 15) {
        unsigned w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = p[2 * i] | ((unsigned)p[2 * i + 1] << 16);
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

// A (M = channel of dz or x, K = pixel) run: channels mg*8 .. +7 of pixel k.
template <int MODE>
__device__ __forceinline__ uint4 wgrad_a8(const Op<MODE> &o, int m, int k, int ke)
{
    const int C = MODE == CONV_WGRAD ? o.g.Cout : o.g.Cin;
    if (k >= ke || m >= o.M) return make_uint4(0, 0, 0, 0);
    if (m + 8 <= o.M && (C & 7) == 0) return ld8(o.a + (long long)k * C + m);
    unsigned short v[8];
    for (int i = 0; i < 8; ++i) v[i] = m + i < o.M ? o.a[(long long)k * C + m + i] : 0;
    return make_uint4(v[0] | ((unsigned)v[1] << 16), v[2] | ((unsigned)v[3] << 16), v[4] | ((unsigned)v[5] << 16),
                      v[6] | ((unsigned)v[7] << 16));
}

// B (N = tap x Cin for conv, child x Cout for upconv; K = pixel) run: n .. n+7 at pixel k.
template <int MODE>
__device__ __forceinline__ uint4 wgrad_b8(const Op<MODE> &o, int n, int k, int ke)
{
    const ConvGeom &g = o.g;
    if (k >= ke || n >= o.N) return make_uint4(0, 0, 0, 0);
    const Pix p = pix(g, k);
    unsigned short v[8];
    const int C = MODE == CONV_WGRAD ? g.Cin : g.Cout;
    const int grp = n / C, c = n - grp * C;
    long long base = -1;
    if (MODE == CONV_WGRAD) {
        const int yy = p.y + grp / 3 - 1, xx = p.x + grp % 3 - 1;
        if (yy >= 0 && yy < g.H && xx >= 0 && xx < g.W) base = (((long long)p.b * g.H + yy) * g.W + xx) * C;
    } else {
        const int Y = 2 * p.y + grp / 2, X = 2 * p.x + (grp & 1);
        base = (((long long)p.b * 2 * g.H + Y) * 2 * g.W + X) * C;
    }
    if ((C & 7) == 0 && n + 8 <= o.N) return base < 0 ? make_uint4(0, 0, 0, 0) : ld8(o.b + base + c);
    for (int i = 0; i < 8; ++i) {   // a run crossing a tap / child boundary or the end of N
        const int ni = n + i;
        v[i] = 0;
        if (ni < o.N) {
            const int gi = ni / C, ci = ni - gi * C;
            long long bi = -1;
            if (MODE == CONV_WGRAD) {
                const int yy = p.y + gi / 3 - 1, xx = p.x + gi % 3 - 1;
                if (yy >= 0 && yy < g.H && xx >= 0 && xx < g.W) bi = (((long long)p.b * g.H + yy) * g.W + xx) * C;
            } else {
                bi = (((long long)p.b * 2 * g.H + 2 * p.y + gi / 2) * 2 * g.W + 2 * p.x + (gi & 1)) * C;
            }
            if (bi >= 0) v[i] = o.b[bi + ci];
        }
    }
    return make_uint4(v[0] | ((unsigned)v[1] << 16), v[2] | ((unsigned)v[3] << 16), v[4] | ((unsigned)v[5] << 16),
                      v[6] | ((unsigned)v[7] << 16));
}

template <int MODE>
__global__ void __launch_bounds__(128) k_gemm_tc(const Op<MODE> o, float *out, int *err)
{
    __shared__ __align__(1024) unsigned char As[TM * TK * 2];
    __shared__ __align__(1024) unsigned char Bs[TN * TK * 2];
    __shared__ unsigned long long bar;
    __shared__ unsigned tmem_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
    const int kb = blockIdx.z * o.klen;
    const int ke = min(kb + o.klen, o.K);
    const unsigned b = tc_smem(&bar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&tmem_sh)),
                     "r"(TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_sh;
    bool ok = true;
    int chunk = 0;
    constexpr bool MN = MODE == CONV_WGRAD || MODE == UP_WGRAD;
    for (int k0 = kb; k0 < ke && ok; k0 += TK, ++chunk) {
        if (MN) {
            // A: TK pixels x TM/8 runs (4 per thread); B: TK pixels x TN/8 runs (2 per thread)
#pragma unroll
            for (int i = 0; i < TK * TM / 8 / 128; ++i) {
                const int t = tid + 128 * i, k = t / (TM / 8), mg = t - k * (TM / 8);
                *reinterpret_cast<uint4 *>(As + tc_off_mn(8 * mg, k)) = wgrad_a8<MODE>(o, m0 + 8 * mg, k0 + k, ke);
            }
#pragma unroll
            for (int i = 0; i < TK * TN / 8 / 128; ++i) {
                const int t = tid + 128 * i, k = t / (TN / 8), ng = t - k * (TN / 8);
                *reinterpret_cast<uint4 *>(Bs + tc_off_mn(8 * ng, k)) = wgrad_b8<MODE>(o, n0 + 8 * ng, k0 + k, ke);
            }
        } else {
            unsigned short seg[16];
#pragma unroll
            for (int h = 0; h < 2; ++h) {          // A: row tid, K halves
                if (m0 + tid < o.M) fillA<MODE>(o, m0 + tid, k0 + 16 * h, ke, seg);
                else
                    for (int i = 0; i < 16; ++i) seg[i] = 0;
                tc_store16(As, tid, 16 * h, seg);
            }
            {                                      // B: row tid % 64, K half tid / 64
                const int r = tid & (TN - 1), h = tid / TN;
                if (n0 + r < o.N) fillB<MODE>(o, n0 + r, k0 + 16 * h, ke, seg);
                else
                    for (int i = 0; i < 16; ++i) seg[i] = 0;
                tc_store16(Bs, r, 16 * h, seg);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // operands visible to the tensor cores
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int ks = 0; ks < TK / 16; ++ks) {
                const unsigned long long ad = tc_desc(tc_smem(As) + ks * 2 * T_LBO);
                const unsigned long long bd = tc_desc(tc_smem(Bs) + ks * 2 * T_LBO);
                const unsigned accum = (chunk > 0 || ks > 0) ? 1u : 0u;
                asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                             "l"(ad), "l"(bd), "r"(MN ? TC_IDESC_MN : TC_IDESC), "r"(accum)
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(b)
                         : "memory");
        }
        ok = __syncthreads_and(tc_wait(b, chunk & 1)) != 0;   // the MMAs have read the operands
    }
    if (!ok) {   // give the outstanding MMAs one more bounded wait before the tensor memory is freed
        if (tid == 0) atomicOr(err, 1);
        tc_wait(b, (chunk - 1) & 1);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float *dst = out + (long long)blockIdx.z * o.M * o.N;
        const int row = m0 + warp * 32 + lane;
#pragma unroll
        for (int c = 0; c < TN; c += 16) {
            unsigned v[16];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                         "%12, %13, %14, %15}, [%16];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                           "=r"(v[14]), "=r"(v[15])
                         : "r"(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < o.M) {
                float *rp = dst + (long long)row * o.N + n0 + c;
                if (n0 + c + 16 <= o.N && (o.N & 3) == 0) {   // 16-byte stores
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4 *>(rp + j) =
                            chunk > 0 ? make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                                                    __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]))
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (n0 + c + j < o.N) rp[j] = chunk > 0 ? __uint_as_float(v[j]) : 0.f;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
}

// ---------------------------------------------------------------------------
// Windowed implicit GEMM of the 3x3 convolutions whose operand channels C
// (forward: C = Cin; data gradient: C = Cout, taps mirrored) are 16 times a
// power of two.  M rows are positions q of the zero-padded pixel grid
// [B][H+2][W+2], flattened (row length Wps = W + 2); output q of tap (ky, kx)
// reads the input at q + s ((ky-1) Wps + (kx-1)), s = +1 / -1, which for an
// interior q stays inside the same image's padded grid.  A CTA computes T
// consecutive 128-row tiles, [q0, q0 + 128 T), so the A operand of every tap
// and tile is one window of the padded input, positions
// [q0 - Wps - 1, q0 + 128 T + Wps + 1), read at a row offset: no im2col
// gather.  Window layout: channel group g (8 channels = 16 bytes) of
// window position p at g GS + 16 p, the K-major core-matrix layout with
// adjacent 8-row groups (SBO 128) and K groups GS apart (LBO GS); a tap's
// operand starts 16 bytes per position further on.  Output rows at padding
// positions are computed and dropped.
//
// K runs over stages of cs channels (all 9 taps each): the stage's window and
// weights [tn][9][cs] (K-major, 8-row groups adjacent, K groups 16 tn bytes
// apart), copied by all threads with cp.async into one of two buffers, each
// with an MMA mbarrier (tcgen05.commit); the copies of stage j+1 run under
// the MMAs of stage j.  One thread issues the T x 9 x cs/16 MMAs (128 x tn x 16) of a
// stage, tiles innermost so that consecutive MMAs feed different
// accumulators in tensor memory.  Large layers split their stages over
// blockIdx.z (FP32 slices, summed by the consumer); otherwise the epilogue
// may apply bias, ReLU and BF16 rounding itself.  (TMA boxes were measured
// slower here: a channel group of a pixel is a 16-byte inner box extent.)
// ---------------------------------------------------------------------------
struct WinOp {
    int B, H, W, C, N;
    int sign;                      // +1 forward, -1 data gradient
    int wps;                       // padded row length W + 2 (positions)
    int T;                         // 128-row tiles per CTA
    int tn, tstride;               // N tile (multiple of 16, <= 256); tensor-memory columns per tile
    int cs, lg_g, spz;             // channels per stage; log2(cs / 8); stages per CTA
    int nw, gs;                    // window positions; bytes between the window's channel groups
    int wbytes, stage_bytes, nbuf; // window bytes; window + weight bytes of a stage; buffers (1 or 2)
    const float *bias;             // fused epilogue (one slice only): y = bf16(relu(acc + bias)), else NULL
    __nv_bfloat16 *y;              //   [B][H][W][N]
};

constexpr int WIN_TN_MAX = 256;
// Threads of the windowed kernels: eight warps share the copies and the
// epilogue (warps w and w + 4 read the same tensor-memory lane quadrant and
// take alternate 16-column chunks); thread 0 issues the MMAs.
constexpr int WT = 256;

__host__ __device__ inline int win_tmem_cols(int cols)
{
    int c = 32;
    while (c < cols) c *= 2;
    return c;
}

__device__ __forceinline__ void cp_async16(unsigned dst, const void *src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(__cvta_generic_to_global(src)),
                 "r"(valid ? 16 : 0)
                 : "memory");
}

// cp.async copies of a window of the padded grid [B][H+2][W+2]: positions
// [q0, q0 + nw) (q0 may be negative), channels [c0, c0 + 8 G) of t
// [B][H][W][C], G = 2^lg_g channel groups; group g of position p at
// base + g gs + 16 p, zeros at the padding.  Thread -> group g = tid % G,
// positions tid / G, + WT / G, ...
__device__ __forceinline__ void copy_window(const unsigned short *t, int B, int H, int W, int C, int c0, int lg_g,
                                            int q0, int nw, int gs, unsigned base)
{
    const int tid = threadIdx.x, Wp = W + 2, Hp = H + 2, G = 1 << lg_g;
    const int g = tid & (G - 1), pstep = WT >> lg_g;
    int p = tid >> lg_g;
    // q = q0 + p, decoded from q + Hp Wp >= 0: padded row ra over the batch
    // (image bi - 1, row py), column px
    const int qq = q0 + p + Hp * Wp;
    const int ra = qq / Wp;
    int px = qq - ra * Wp;
    int bi = ra / Hp, py = ra - bi * Hp;
    for (; p < nw; p += pstep) {
        const bool valid = bi >= 1 && bi <= B && py >= 1 && py <= H && px >= 1 && px <= W;
        const unsigned short *src = valid ? t + ((long long)((bi - 1) * H + py - 1) * W + px - 1) * C + c0 + 8 * g : t;
        cp_async16(base + g * gs + p * 16, src, valid);
        px += pstep;
        while (px >= Wp) {
            px -= Wp;
            if (++py == Hp) {
                py = 0;
                ++bi;
            }
        }
    }
}

// The CTA copies stage s (channels [s cs, (s+1) cs)) into the buffer at base
// with cp.async (16 bytes each, zero fill at the padding) and commits them as
// one group: the window positions [q0 - Wps - 1, q0 + 128 T + Wps + 1) of the
// padded grid (thread -> channel group fastest, then positions; each thread
// keeps its current row's pixel pointer and steps through the positions
// without division), then the weights (thread -> row fastest, K group next).
__device__ __forceinline__ void win_copy_stage(const WinOp &o, const unsigned short *t, const unsigned short *w,
                                               int q0, int n0, int s, unsigned base)
{
    const int tid = threadIdx.x, G = 1 << o.lg_g, KG = 9 * G, Hp = o.H + 2, Wps = o.wps;
    const int c0 = s * o.cs;
    {
        const int g = tid & (G - 1), pstep = WT >> o.lg_g;
        int p = tid >> o.lg_g;
        // grid position q = q0 - Wps - 1 + p, decoded once from q + Hp Wps >= 0 as
        // (image bi - 1, padded row py, column x), then stepped without division
        const int qq = q0 - Wps - 1 + p + Hp * Wps, ra = qq / Wps;
        int x = qq - ra * Wps, bi = ra / Hp, py = ra - bi * Hp;
        auto row_ptr = [&]() -> const unsigned short * {   // pixel (row, column x) at + x C
            return (bi >= 1 && bi <= o.B && py >= 1 && py <= o.H)
                       ? t + ((long long)(bi - 1) * o.H + py - 1) * o.W * o.C + c0 + 8 * g - o.C
                       : nullptr;
        };
        const unsigned short *rp = row_ptr();
        const unsigned dst0 = base + g * o.gs;
        for (; p < o.nw; p += pstep) {
            const bool valid = rp && x >= 1 && x <= o.W;
            cp_async16(dst0 + p * 16, valid ? rp + (long long)x * o.C : t, valid);
            x += pstep;
            if (x >= Wps) {
                do {
                    x -= Wps;
                    if (++py == Hp) {
                        py = 0;
                        ++bi;
                    }
                } while (x >= Wps);
                rp = row_ptr();
            }
        }
    }
    {   // weights: item (row r, K group kg = tap G + cg) -> base + wbytes + kg 16 tn + 16 r.  A warp
        // takes 8 rows x 4 K groups: each row gives 64 contiguous bytes (two whole sectors), and
        // each 8-thread store phase 128 contiguous bytes of shared memory.
        const unsigned wb = base + o.wbytes;
        const int K = 9 * o.C, lane = tid & 31, rl = lane & 7, kl = lane >> 3;
        const int nrt = o.tn / 8, nkt = (KG + 3) / 4;
        // tile (row tile rt, K tile kt) = warp, + 8, ... in row-tile-fastest order, stepped without division
        int kt = 0, rt = tid >> 5;
        while (rt >= nrt) {
            rt -= nrt;
            ++kt;
        }
        for (; kt < nkt;) {
            const int r = rt * 8 + rl, kg = kt * 4 + kl, n = n0 + r;
            if (kg < KG) {
                const bool valid = n < o.N;
                cp_async16(wb + kg * o.tn * 16 + r * 16,
                           valid ? w + (long long)n * K + (kg >> o.lg_g) * o.C + c0 + 8 * (kg & (G - 1)) : w, valid);
            }
            rt += WT / 32;
            while (rt >= nrt) {
                rt -= nrt;
                ++kt;
            }
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// One 128 x N x 16 MMA into tensor memory; the accumulate flag is an immediate
// (ACC 0: D = A B, 1: D += A B), so the issue loop spends no predicate set-up.
template <int ACC>
__device__ __forceinline__ void mma_f16(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc)
{
    if (ACC)
        asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;" ::"r"(d), "l"(a), "l"(b), "r"(idesc)
                     : "memory");
    else
        asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 0;" ::"r"(d), "l"(a), "l"(b), "r"(idesc)
                     : "memory");
}

// The T tiles of one (tap, 16-channel) step: tile t's A starts 128 rows (128 in
// 16-byte units) further on, its accumulator T_STRIDE columns further on.
template <int T, int ACC>
__device__ __forceinline__ void mma_tiles(unsigned tmem, int tstride, unsigned long long ad, unsigned long long bd,
                                          unsigned idesc)
{
#pragma unroll
    for (int tt = 0; tt < T; ++tt) mma_f16<ACC>(tmem + (unsigned)(tt * tstride), ad + (unsigned long long)(tt * 128), bd, idesc);
}

template <int T>
__global__ void __launch_bounds__(WT, 2) k_conv_win(const WinOp o, const unsigned short *t, const unsigned short *w,
                                                 float *out, int *err)
{
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ unsigned long long bars[2];
    __shared__ unsigned tmem_sh;
    __shared__ float bias_sh[WIN_TN_MAX];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, half = warp >> 2;   // tensor-memory lane quadrant; column-chunk parity
    const int Wps = o.wps, Hp = o.H + 2, G = 1 << o.lg_g;
    const int q0 = blockIdx.x * (T * TM), n0 = blockIdx.y * o.tn, s0 = blockIdx.z * o.spz;
    const int ns = min(o.spz, o.C / o.cs - s0);   // stages of this CTA
    const int tcols = win_tmem_cols(T * o.tstride);
    const unsigned sm0 = tc_smem(dsm);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&tmem_sh)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < 2; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&bars[i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (o.y)
        for (int i = tid; i < o.tn; i += WT) bias_sh[i] = o.bias[min(n0 + i, o.N - 1)];
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_sh;
    win_copy_stage(o, t, w, q0, n0, s0, sm0);
    const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(o.tn >> 3) << 17) |
                           ((unsigned)(TM >> 4) << 24);
    bool ok = true;
    int issued = 0;   // stages whose MMAs were issued (stage j commits to bars[j % nbuf])
    for (int s = 0; s < ns && ok; ++s) {
        const int b = s % o.nbuf;
        if (o.nbuf == 2 && s + 1 < ns) {   // copy stage s + 1 under the MMAs of stage s
            if (s >= 1)   // the MMAs of stage s - 1 have read the other buffer
                ok = __syncthreads_and(tc_wait(tc_smem(&bars[(s - 1) & 1]), ((s - 1) >> 1) & 1)) != 0;
            if (!ok) break;
            win_copy_stage(o, t, w, q0, n0, s0 + s + 1, sm0 + ((s + 1) & 1) * o.stage_bytes);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the copies visible to the tensor cores
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned base = sm0 + b * o.stage_bytes;
            const unsigned long long dA = (unsigned long long)((2 * o.gs) >> 4);   // 16 channels further on
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const int ky = tap / 3, kx = tap % 3;
                const int r0 = o.sign * ((ky - 1) * Wps + (kx - 1)) + Wps + 1;   // window row of tile 0, row 0
                // descriptors of the slice's first 16 channels, advanced per 16 channels:
                // A by two channel groups (2 gs bytes), B by two K groups (32 tn bytes);
                // tile t's A starts 128 rows (2048 bytes) further on.  The tiles are
                // the innermost loop, so consecutive MMAs feed different accumulators.
                unsigned long long ad = tc_desc(base + r0 * 16, o.gs, 128);
                unsigned long long bd = tc_desc(base + o.wbytes + tap * G * o.tn * 16, o.tn * 16, 128);
                const unsigned long long dB = (unsigned long long)((2 * o.tn * 16) >> 4);
                int j = 0;
                if (s == 0 && tap == 0) {   // the first step of each accumulator overwrites it
                    mma_tiles<T, 0>(tmem, o.tstride, ad, bd, idesc);
                    ad += dA;
                    bd += dB;
                    j = 1;
                }
                for (; j < o.cs / 16; ++j) {
                    mma_tiles<T, 1>(tmem, o.tstride, ad, bd, idesc);
                    ad += dA;
                    bd += dB;
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             tc_smem(&bars[b]))
                         : "memory");
        }
        issued = s + 1;
        if (o.nbuf == 1 && s + 1 < ns) {   // one buffer: the MMAs of stage s read it before the next copies
            ok = __syncthreads_and(tc_wait(tc_smem(&bars[0]), s & 1)) != 0;
            if (ok) win_copy_stage(o, t, w, q0, n0, s0 + s + 1, sm0);
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (issued > 0) {   // the last issued stage's commit covers every earlier MMA
        const int l = issued - 1;
        const bool done = tc_wait(tc_smem(&bars[l % o.nbuf]), (l / o.nbuf) & 1);
        ok = __syncthreads_and(ok && done) != 0;
    }
    if (!ok) {
        if (tid == 0) atomicOr(err, 1);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float *dst = out + (long long)blockIdx.z * o.B * o.H * o.W * o.N;
        for (int t = 0; t < T; ++t) {
            const int q = q0 + t * TM + quad * 32 + lane;
            const int ra = q / Wps, px = q - ra * Wps, bi = ra / Hp, py = ra - bi * Hp;
            const long long pixel = (bi < o.B && py >= 1 && py <= o.H && px >= 1 && px <= o.W)
                                        ? ((long long)bi * o.H + py - 1) * o.W + px - 1
                                        : -1;
            for (int c = 16 * half; c < o.tn; c += 32) {
                unsigned v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                    "%12, %13, %14, %15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(tmem + ((unsigned)(quad * 32) << 16) + (unsigned)(t * o.tstride + c)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (pixel >= 0 && o.y) {   // bias, ReLU, BF16 (round to nearest even)
                    __nv_bfloat16 *yp = o.y + pixel * o.N + n0 + c;
                    unsigned short h[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        h[j] = __bfloat16_as_ushort(__float2bfloat16_rn(fmaxf(__uint_as_float(v[j]) + bias_sh[c + j], 0.f)));
                    if (n0 + c + 16 <= o.N && (o.N & 7) == 0) {   // 16-byte stores
                        reinterpret_cast<uint4 *>(yp)[0] =
                            make_uint4(h[0] | ((unsigned)h[1] << 16), h[2] | ((unsigned)h[3] << 16),
                                       h[4] | ((unsigned)h[5] << 16), h[6] | ((unsigned)h[7] << 16));
                        reinterpret_cast<uint4 *>(yp)[1] =
                            make_uint4(h[8] | ((unsigned)h[9] << 16), h[10] | ((unsigned)h[11] << 16),
                                       h[12] | ((unsigned)h[13] << 16), h[14] | ((unsigned)h[15] << 16));
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (n0 + c + j < o.N) yp[j] = __ushort_as_bfloat16(h[j]);
                    }
                } else if (pixel >= 0) {
                    float *rp = dst + pixel * o.N + n0 + c;
                    if (n0 + c + 16 <= o.N && (o.N & 3) == 0) {   // 16-byte stores
#pragma unroll
                        for (int j = 0; j < 16; j += 4)
                            *reinterpret_cast<float4 *>(rp + j) =
                                make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                                            __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (n0 + c + j < o.N) rp[j] = __uint_as_float(v[j]);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

// Launch geometry of the windowed kernel for C operand channels and N
// outputs; false when it does not apply (C not 16 times a power of two, an
// unaligned operand, or sizes beyond its limits).
struct WinPlan {
    WinOp o;
    const unsigned short *t, *w;   // input [B][H][W][C], weights [N][9][C] (raw BF16 bits)
    dim3 grid;
    size_t smem;
};

int win_smem_limit()
{
    static int lim = -1;
    if (lim < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) lim = 0;
        lim -= 4096;   // the kernel's static shared memory and the alignment of the dynamic block
        if (lim > 0 && (cudaFuncSetAttribute(k_conv_win<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess ||
                        cudaFuncSetAttribute(k_conv_win<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess ||
                        cudaFuncSetAttribute(k_conv_win<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess))
            lim = 0;
    }
    return lim;
}

int win_sm_count()
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    }
    return sms;
}

// Stage geometry for T tiles and cs channels: window positions, group
// stride and bytes.  The group stride is padded so that the 8 threads of a
// 16-byte store phase (consecutive groups, then positions) hit distinct bank
// quads; every operand offset stays a multiple of 16 bytes.
void win_stage(WinOp &o, int T, int cs)
{
    const int G = cs / 8;
    o.T = T;
    o.cs = cs;
    o.lg_g = 0;
    while ((1 << o.lg_g) < G) ++o.lg_g;
    o.nw = T * TM + 2 * o.wps + 2;
    const int step = G >= 8 ? 1 : 8 / G;
    o.gs = ((o.nw + 7) / 8 * 8 + step) * 16;
    o.wbytes = G * o.gs;
    o.stage_bytes = o.wbytes + o.tn * 9 * cs * 2;
}

// max_splits bounds blockIdx.z (the FP32 slices the caller can hold).
bool win_plan(const __nv_bfloat16 *t, const __nv_bfloat16 *w, ConvGeom g, int C, int N, int sign, int max_splits,
              WinPlan &wp)
{
    if (C < 16 || C % 16 != 0 || ((C / 16) & (C / 16 - 1)) != 0 || N < 1 || C > 1024 || g.W < 1 ||
        g.H < 1 || g.B < 1 || (reinterpret_cast<uintptr_t>(t) & 15) != 0 || (reinterpret_cast<uintptr_t>(w) & 15) != 0)
        return false;
    const int lim = win_smem_limit(), sms = win_sm_count();
    constexpr int kStageCap = 100 * 1024;   // one stage; two buffers stay below the shared-memory limit
    WinOp &o = wp.o;
    o.B = g.B, o.H = g.H, o.W = g.W, o.C = C, o.N = N, o.sign = sign;
    o.wps = g.W + 2;
    const long long Q = (long long)g.B * (g.H + 2) * o.wps;
    if (Q + 8LL * TM + 4LL * o.wps > INT_MAX / 2) return false;
    o.bias = nullptr;
    o.y = nullptr;
    o.tn = std::min(WIN_TN_MAX, (N + 15) / 16 * 16);
    o.tstride = win_tmem_cols(o.tn);
    const int ntn = (N + o.tn - 1) / o.tn;
    // Four tiles per CTA where the tensor memory allows: an MMA costs the same for
    // any N, so the tiles share each stage's weights (the deep layers' copies are
    // mostly weights); the channel stage shrinks until two buffers fit, and the
    // stages split over CTAs (blockIdx.z) while the grid has fewer CTAs than SMs.
    int T = 0, cs = C;
    for (int cand : {4, 2, 1}) {
        if (cand * o.tstride > 512) continue;
        int c = C;
        for (win_stage(o, cand, c); c > 16 && (o.stage_bytes > kStageCap || (C / c > 1 && 2 * o.stage_bytes > lim));
             win_stage(o, cand, c))
            c /= 2;
        if ((C / c > 1 ? 2 : 1) * o.stage_bytes <= lim) {
            T = cand;
            cs = c;
            break;
        }
    }
    if (T == 0) return false;
    const int nstages = C / cs;
    o.nbuf = nstages > 1 ? 2 : 1;
    win_stage(o, T, cs);
    if (o.nbuf * o.stage_bytes > lim || o.gs >= (1 << 18)) return false;
    const long long xt = (Q + T * TM - 1) / (T * TM);
    int z = 1;
    while (xt * ntn * z < sms && z * 2 <= nstages && z * 2 <= max_splits) z *= 2;
    o.spz = nstages / z;
    wp.grid = dim3((unsigned)xt, (unsigned)ntn, (unsigned)z);
    wp.smem = (size_t)o.nbuf * o.stage_bytes;
    wp.t = reinterpret_cast<const unsigned short *>(t);
    wp.w = reinterpret_cast<const unsigned short *>(w);
    return true;
}

// Returns the FP32 slices written (blockIdx.z extent).
int win_launch(const WinPlan &wp, float *out, cudaStream_t st)
{
    count_launch();
    auto kern = wp.o.T == 4 ? k_conv_win<4> : wp.o.T == 2 ? k_conv_win<2> : k_conv_win<1>;
    kern<<<wp.grid, WT, wp.smem, st>>>(wp.o, wp.t, wp.w, out, unet_error_word());
    return (int)wp.grid.z;
}

// ---------------------------------------------------------------------------
// Windowed weight gradient of the 3x3 convolutions (Cin a multiple of 16,
// Cout of 8):  dW[co][tap][ci] = sum over positions q of the padded grid of
// dz[q][co] x[q + (ky-1)(W+2) + (kx-1)][ci], dz read as zero at the padding
// positions.  K = positions; per tap one MMA with M = 128 output channels
// (A = dz, MN-major) and N = a slice of ncs input channels (B = the input
// window of the forward kernel read at the tap's row offset, MN-major:
// position rows 16 bytes apart, channel groups GS apart).  The dz tile keeps
// the channel groups of 8 positions adjacent (SBO 128, K groups ga 128 bytes
// apart), so the MMA rows above Cout read the next positions' data (dropped
// rows of D) inside a 2 KB pad.  The nine accumulators sit in tensor memory.
// A CTA takes a span of positions in stages of pb (dz tile + window by
// cp.async, two buffers) and writes its FP32 partial [Cout][9][Cin] slice;
// the spans are the K splits, summed by the consumer.
// ---------------------------------------------------------------------------
struct WgOp {
    const unsigned short *dz, *x;   // [B][H][W][Cout], [B][H][W][Cin] (raw BF16 bits)
    int B, H, W, Cin, Cout;
    int ncs, lg_gx, tstride;        // input channels per CTA (N); log2(ncs / 8); tensor-memory columns per tap
    int ga;                         // output-channel groups of a full M tile (<= 16; the last tile may have fewer)
    int pb, span;                   // positions per stage (multiple of 16); per CTA (multiple of pb)
    int nw, gs;                     // window positions (pb + 2 (W+2) + 2); bytes between its channel groups
    int abytes, stage_bytes;        // dz tile bytes (with the pad); dz tile + window bytes
};

// ga = output-channel groups of this CTA's M tile
__device__ __forceinline__ void wg_load_stage(const WgOp &o, int p0, int m0, int ga, int c0, unsigned base)
{
    const int tid = threadIdx.x, Wp = o.W + 2, Hp = o.H + 2;
    // dz tile: position k, channel group g at (k >> 3) ga 128 + g 128 + (k & 7) 16; thread -> (k, g), g fastest
    if ((ga & (ga - 1)) == 0) {   // ga a power of two: g fixed per thread, positions stepped without division
        int lg = 0;
        while ((1 << lg) < ga) ++lg;
        const int g = tid & (ga - 1), kstep = WT >> lg;
        int k = tid >> lg;
        const int q = p0 + k, ra = q / Wp;
        int px = q - ra * Wp, bi = ra / Hp, py = ra - bi * Hp;
        for (; k < o.pb; k += kstep) {
            const bool valid = bi < o.B && py >= 1 && py <= o.H && px >= 1 && px <= o.W;
            const unsigned short *src =
                valid ? o.dz + ((long long)(bi * o.H + py - 1) * o.W + px - 1) * o.Cout + m0 + 8 * g : o.dz;
            cp_async16(base + (k >> 3) * (ga * 128) + g * 128 + (k & 7) * 16, src, valid);
            px += kstep;
            while (px >= Wp) {
                px -= Wp;
                if (++py == Hp) {
                    py = 0;
                    ++bi;
                }
            }
        }
    } else {
        for (int i = tid; i < o.pb * ga; i += WT) {
            const int k = i / ga, g = i - k * ga;
            const int q = p0 + k;
            const int ra = q / Wp, px = q - ra * Wp, bi = ra / Hp, py = ra - bi * Hp;
            const bool valid = bi < o.B && py >= 1 && py <= o.H && px >= 1 && px <= o.W;
            const unsigned short *src =
                valid ? o.dz + ((long long)(bi * o.H + py - 1) * o.W + px - 1) * o.Cout + m0 + 8 * g : o.dz;
            cp_async16(base + (k >> 3) * (ga * 128) + g * 128 + (k & 7) * 16, src, valid);
        }
    }
    copy_window(o.x, o.B, o.H, o.W, o.Cin, c0, o.lg_gx, p0 - Wp - 1, o.nw, o.gs, base + o.abytes);
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__global__ void __launch_bounds__(WT, 1) k_wgrad_win(const WgOp o, float *out, int *err)
{
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ unsigned long long bars[2];
    __shared__ unsigned tmem_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, half = warp >> 2;   // tensor-memory lane quadrant; column-chunk parity
    const int Wp = o.W + 2;
    const int Q = o.B * (o.H + 2) * Wp;
    const int pbeg = blockIdx.x * o.span, pend = min(pbeg + o.span, Q);
    const int c0 = blockIdx.y * o.ncs, m0 = blockIdx.z * 128, ga = min(o.ga, (o.Cout - m0) >> 3);
    const int ns = (pend - pbeg + o.pb - 1) / o.pb;
    const int tcols = win_tmem_cols(9 * o.tstride);
    const unsigned sm0 = tc_smem(dsm);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&tmem_sh)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&bars[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&bars[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (ns > 0) wg_load_stage(o, pbeg, m0, ga, c0, sm0);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_sh;
    const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                           ((unsigned)(o.ncs >> 3) << 17) | ((unsigned)(TM >> 4) << 24);
    const int lbo_a = ga * 128;
    bool ok = true;
    int issued = 0;
    for (int s = 0; s < ns && ok; ++s) {
        const int b = s & 1;
        if (s + 1 < ns) {
            if (s >= 1)   // the MMAs of stage s - 1 have read the other buffer
                ok = __syncthreads_and(tc_wait(tc_smem(&bars[(s - 1) & 1]), ((s - 1) >> 1) & 1)) != 0;
            if (!ok) break;
            wg_load_stage(o, pbeg + (s + 1) * o.pb, m0, ga, c0, sm0 + ((s + 1) & 1) * o.stage_bytes);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the copies visible to the tensor cores
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned abase = sm0 + b * o.stage_bytes, xbase = abase + o.abytes;
            // descriptors of K step 0, advanced per step: A by 16 positions (2 lbo_a bytes),
            // B by 16 window rows (256 bytes); the address field stays below 256 KB
            unsigned long long ad = tc_desc(abase, lbo_a, 128), bd[9];
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) bd[tap] = tc_desc(xbase + ((tap / 3) * Wp + tap % 3) * 16, 128, o.gs);
            const unsigned long long dA = (unsigned long long)((2 * lbo_a) >> 4);
            int kk = 0;
            if (s == 0) {   // the first K step overwrites the nine accumulators
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    mma_f16<0>(tmem + (unsigned)(tap * o.tstride), ad, bd[tap], idesc);
                    bd[tap] += 16;
                }
                ad += dA;
                kk = 1;
            }
            for (; kk < o.pb / 16; ++kk) {
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    mma_f16<1>(tmem + (unsigned)(tap * o.tstride), ad, bd[tap], idesc);
                    bd[tap] += 16;
                }
                ad += dA;
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             tc_smem(&bars[b]))
                         : "memory");
        }
        issued = s + 1;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (issued > 0) {   // the last issued stage's commit covers every earlier MMA
        const int l = issued - 1;
        const bool done = tc_wait(tc_smem(&bars[l & 1]), (l >> 1) & 1);
        ok = __syncthreads_and(ok && done) != 0;
    }
    if (!ok) {
        if (tid == 0) atomicOr(err, 1);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int co = m0 + quad * 32 + lane;
        float *dst = out + ((long long)blockIdx.x * o.Cout + co) * 9 * o.Cin + c0;
        const int nch = o.ncs / 16;   // 16-column chunks per tap; chunk index tap nch + c / 16, by parity
        for (int ci = half; ci < 9 * nch; ci += 2) {
            const int tap = ci / nch, c = (ci - tap * nch) * 16;
            {
                unsigned v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                    "%12, %13, %14, %15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(tmem + ((unsigned)(quad * 32) << 16) + (unsigned)(tap * o.tstride + c)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (co < o.Cout && ns > 0) {
                    float *rp = dst + tap * o.Cin + c;
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4 *>(rp + j) =
                            make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]), __uint_as_float(v[j + 2]),
                                        __uint_as_float(v[j + 3]));
                } else if (co < o.Cout) {   // an empty span: a zero slice
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4 *>(dst + tap * o.Cin + c + j) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

struct WgPlan {
    WgOp o;
    dim3 grid;
    size_t smem;
};

// false when the windowed weight gradient does not apply; max_splits bounds
// the position spans (FP32 slices [Cout][9][Cin] the caller can hold).
bool wg_plan(const __nv_bfloat16 *dz, const __nv_bfloat16 *x, ConvGeom g, int max_splits, WgPlan &wp)
{
    const int Cin = g.Cin, Cout = g.Cout;
    if (Cin < 16 || Cin % 16 != 0 || Cout < 8 || Cout % 8 != 0 || Cin > 4096 || max_splits < 1 ||
        (reinterpret_cast<uintptr_t>(dz) & 15) != 0 || (reinterpret_cast<uintptr_t>(x) & 15) != 0 ||
        (long long)g.B * (g.H + 2) * (g.W + 2) + 2048LL > INT_MAX / 2)
        return false;
    const int lim = win_smem_limit(), sms = win_sm_count();
    WgOp &o = wp.o;
    o.dz = reinterpret_cast<const unsigned short *>(dz);
    o.x = reinterpret_cast<const unsigned short *>(x);
    o.B = g.B, o.H = g.H, o.W = g.W, o.Cin = Cin, o.Cout = Cout;
    o.ncs = Cin % 32 == 0 ? 32 : 16;
    o.lg_gx = o.ncs == 32 ? 2 : 1;
    o.tstride = o.ncs;
    o.ga = std::min(16, Cout / 8);
    const int Wp = g.W + 2;
    for (o.pb = 512; o.pb >= 32; o.pb -= 32) {
        o.nw = o.pb + 2 * Wp + 2;
        const int G = o.ncs / 8, step = G >= 8 ? 1 : 8 / G;
        o.gs = ((o.nw + 7) / 8 * 8 + step) * 16;
        o.abytes = o.pb * o.ga * 16 + 2048;
        o.stage_bytes = o.abytes + G * o.gs;
        if (2 * o.stage_bytes <= lim && o.gs < (1 << 18)) break;
    }
    if (o.pb < 32) return false;
    const long long Q = (long long)g.B * (g.H + 2) * Wp;
    const int cols = Cin / o.ncs, mt = (Cout + 127) / 128;
    // spans: about one CTA per SM (nine accumulators take the tensor memory), whole stages each
    long long spans = std::max(1LL, std::min<long long>((Q + o.pb - 1) / o.pb, (sms + cols * mt - 1) / (cols * mt)));
    spans = std::min<long long>(spans, max_splits);
    const long long stages = ((Q + spans - 1) / spans + o.pb - 1) / o.pb;
    o.span = (int)(stages * o.pb);
    wp.grid = dim3((unsigned)((Q + o.span - 1) / o.span), (unsigned)cols, (unsigned)mt);
    wp.smem = (size_t)2 * o.stage_bytes;
    return true;
}

int wg_launch(const WgPlan &wp, float *out, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_wgrad_win, cudaFuncAttributeMaxDynamicSharedMemorySize, win_smem_limit());
        attr = true;
    }
    count_launch();
    k_wgrad_win<<<wp.grid, WT, wp.smem, st>>>(wp.o, out, unet_error_word());
    return (int)wp.grid.x;
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
    dim3 grid((M + TM - 1) / TM, (N + TN - 1) / TN, splits);
    count_launch();
    k_gemm_tc<MODE><<<grid, 128, 0, st>>>(o, out, unet_error_word());
    return splits;
}

}  // namespace unet

using namespace unet;

// ---------------------------------------------------------------------------
// launchers used by the U-Net runtime (unet.cu)
// ---------------------------------------------------------------------------

// FP32 GEMM results for one operation, [splits][M][N] (the caller sums the
// slices); max_splits / out_cap bound the slices; each returns the number used.
// unet_conv3_fwd with bias and y may instead write y = bf16(relu(conv + bias))
// itself, and then returns 0.
int unet_conv3_fwd(const __nv_bfloat16 *x, const __nv_bfloat16 *w, int B, int H, int W, int Cin, int Cout,
                    const float *bias, __nv_bfloat16 *y, float *out, long long out_cap, cudaStream_t st)
{
    ConvGeom g{B, H, W, Cin, Cout};
    const int sms = win_sm_count();
    const long long M = (long long)B * H * W, N = Cout;
    const long long cap = std::max(1LL, out_cap / (M * N));
    WinPlan wp;
    if (win_plan(x, w, g, Cin, Cout, 1, (int)std::min<long long>(cap, 64), wp)) {
        if (bias && y && wp.grid.z == 1) {   // one slice: the epilogue writes y itself
            wp.o.bias = bias;
            wp.o.y = y;
            win_launch(wp, out, st);
            return 0;
        }
        return win_launch(wp, out, st);
    }
    // split K when the output tiles alone leave SMs idle (deep levels, small batches)
    const long long tiles = ((M + TM - 1) / TM) * ((N + TN - 1) / TN);
    long long splits = (2LL * sms + tiles - 1) / tiles;
    splits = std::max(1LL, std::min(splits, cap));
    return gemm<CONV_FWD>(x, w, g, (int)M, Cout, 9 * Cin, (int)splits, out, st);
}

int unet_conv3_dgrad(const __nv_bfloat16 *dz, const __nv_bfloat16 *wt, int B, int H, int W, int Cin, int Cout,
                      float *out, long long out_cap, cudaStream_t st)
{
    ConvGeom g{B, H, W, Cin, Cout};
    const long long cap = std::max(1LL, out_cap / ((long long)B * H * W * Cin));
    WinPlan wp;
    if (win_plan(dz, wt, g, Cout, Cin, -1, (int)std::min<long long>(cap, 64), wp)) return win_launch(wp, out, st);
    return gemm<CONV_DGRAD>(dz, wt, g, B * H * W, Cin, 9 * Cout, 1, out, st);
}

int unet_conv3_wgrad(const __nv_bfloat16 *dz, const __nv_bfloat16 *x, int B, int H, int W, int Cin, int Cout,
                      int max_splits, float *out, cudaStream_t st)
{
    ConvGeom g{B, H, W, Cin, Cout};
    WgPlan wp;
    if (wg_plan(dz, x, g, max_splits, wp)) return wg_launch(wp, out, st);
    const int P = B * H * W;   // gathered: K splits of about 512 pixels
    return gemm<CONV_WGRAD>(dz, x, g, Cout, 9 * Cin, P, std::min(max_splits, std::max(1, P / 512)), out, st);
}

// wt: the upconv weights transposed, [4 Cout][Cin]
int unet_up_fwd(const __nv_bfloat16 *x, const __nv_bfloat16 *wt, int B, int H, int W, int Cin, int Cout,
                 float *out, cudaStream_t st)
{
    ConvGeom g{B, H, W, Cin, Cout};
    return gemm<UP_FWD>(x, wt, g, B * H * W, 4 * Cout, Cin, 1, out, st);
}

int unet_up_dgrad(const __nv_bfloat16 *dy, const __nv_bfloat16 *w, int B, int H, int W, int Cin, int Cout,
                   float *out, cudaStream_t st)
{
    ConvGeom g{B, H, W, Cin, Cout};
    return gemm<UP_DGRAD>(dy, w, g, B * H * W, Cin, 4 * Cout, 1, out, st);
}

int unet_up_wgrad(const __nv_bfloat16 *x, const __nv_bfloat16 *dy, int B, int H, int W, int Cin, int Cout,
                   int max_splits, float *out, cudaStream_t st)
{
    ConvGeom g{B, H, W, Cin, Cout};
    const int P = B * H * W;   // K splits of about 512 input pixels
    return gemm<UP_WGRAD>(x, dy, g, Cin, 4 * Cout, P, std::min(max_splits, std::max(1, P / 512)), out, st);
}

}  // namespace aafwi
