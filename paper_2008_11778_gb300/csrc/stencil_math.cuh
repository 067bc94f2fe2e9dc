// stencil_math.cuh -- the arithmetic of one grid-point update of the
// leap-frog scheme (Sec. 2.2, eq. FWD; the adjoint, eq. FWI_adj, and the
// Born step, eq. Born, are built from the same pieces), shared by every
// step kernel so that all engines compute each cell with the same
// operations in the same order and agree bitwise.
//
//   S(f) = sum_k A_k [(f_{-k} - f_0) + (f_{+k} - f_0)],
//          A = 5040 x (8/5, -1/5, 8/315, -1/560) = (8064, -1008, 128, -9),
//          accumulated k = 4..1 (integer weights: exact in FP32, and no
//          cancellation of a centre weight against the neighbours; the
//          dominant k = 1 term enters last through an fma)
//   T    = rz S_z + S_x  (= 5040 dx^2 L f, rz = dx^2 / dz^2)
//   dG   = 1 - G = dz + dx - dz dx  (Cerjan sponge, from per-row and
//          per-column tables; handled as its negative ndG)
//   f'   = G (2 f - G f_prev + (Wh + Wl) T), evaluated as
//          gp = f_prev - dG f_prev;  t = ((f - gp) + f) + (Wh T + Wl T);
//          f' = t - dG t
//
// Every rounding is explicit (round-to-nearest intrinsics, nothing left to
// the compiler's contraction), and two adjacent cells go through one packed
// FP32x2 instruction (sm_100 and later: __fadd2_rn, __ffma2_rn, __fmul2_rn
// round each lane exactly as the scalar instruction does).  a - c is formed
// as fma(c, -1, a), which is the same rounded value.
#pragma once
#include <cuda_runtime.h>

namespace aafwi {

constexpr float A1 = 8064.f;
constexpr float A2 = -1008.f;
constexpr float A3 = 128.f;
constexpr float A4 = -9.f;

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 cat2(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ float4 neg4(float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }

// (a - c) + (b - c), two cells
__device__ __forceinline__ float2 dd2(float2 c, float2 a, float2 b)
{
    const float2 m1 = bc2(-1.f);
    return __fadd2_rn(__ffma2_rn(c, m1, a), __ffma2_rn(c, m1, b));
}

// A1 d1 + A2 d2 + A3 d3 + A4 d4 for two cells, accumulated from the
// smallest weight up so that the dominant term A1 d1 enters last, unrounded,
// through the final fma
__device__ __forceinline__ float2 wsum2(float2 d1, float2 d2, float2 d3, float2 d4)
{
    float2 s = __fmul2_rn(bc2(A4), d4);
    s = __ffma2_rn(bc2(A3), d3, s);
    s = __ffma2_rn(bc2(A2), d2, s);
    return __ffma2_rn(bc2(A1), d1, s);
}

// T = rz S_z + S_x for the float4 group M (4 adjacent cells of a row); L, R
// the groups to its left and right, up[k-1] / dn[k-1] the groups k rows
// above / below (zeros outside the grid).  The x neighbours of a cell pair
// do not all sit in adjacent registers: the compiler pairs them by moves.
__device__ __forceinline__ float4 stencil_T(float4 L, float4 M, float4 R, const float4 (&up)[4],
                                            const float4 (&dn)[4], float rz)
{
    const float v[12] = {L.x, L.y, L.z, L.w, M.x, M.y, M.z, M.w, R.x, R.y, R.z, R.w};
    float2 sx[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {   // cells (2p, 2p+1)
        const int i = 4 + 2 * p;
        const float2 c = make_float2(v[i], v[i + 1]);
        sx[p] = wsum2(dd2(c, make_float2(v[i - 1], v[i]), make_float2(v[i + 1], v[i + 2])),
                      dd2(c, make_float2(v[i - 2], v[i - 1]), make_float2(v[i + 2], v[i + 3])),
                      dd2(c, make_float2(v[i - 3], v[i - 2]), make_float2(v[i + 3], v[i + 4])),
                      dd2(c, make_float2(v[i - 4], v[i - 3]), make_float2(v[i + 4], v[i + 5])));
    }
    const float2 r2 = bc2(rz);
    const float2 c0 = lo2(M), c1 = hi2(M);
    const float2 s0 = wsum2(dd2(c0, lo2(up[0]), lo2(dn[0])), dd2(c0, lo2(up[1]), lo2(dn[1])),
                            dd2(c0, lo2(up[2]), lo2(dn[2])), dd2(c0, lo2(up[3]), lo2(dn[3])));
    const float2 s1 = wsum2(dd2(c1, hi2(up[0]), hi2(dn[0])), dd2(c1, hi2(up[1]), hi2(dn[1])),
                            dd2(c1, hi2(up[2]), hi2(dn[2])), dd2(c1, hi2(up[3]), hi2(dn[3])));
    return cat2(__ffma2_rn(r2, s0, sx[0]), __ffma2_rn(r2, s1, sx[1]));
}

// -(1 - G) = dz dx - (dz + dx) for the four cells of a group: dz of the row,
// dx and ndx = -dx of the columns.
__device__ __forceinline__ float4 neg_sponge4(float dz, float4 dx, float4 ndx)
{
    const float2 d = bc2(dz), m1 = bc2(-1.f);
    return cat2(__ffma2_rn(d, lo2(dx), __ffma2_rn(d, m1, lo2(ndx))),
                __ffma2_rn(d, hi2(dx), __ffma2_rn(d, m1, hi2(ndx))));
}

// f' = G (2 f - G f_prev + (Wh + Wl) T) for two cells, ndG = -(1 - G)
__device__ __forceinline__ float2 leap2(float2 ndG, float2 cur, float2 prev, float2 T, float2 wh, float2 wl)
{
    const float2 wq = __ffma2_rn(wh, T, __fmul2_rn(wl, T));
    const float2 gp = __ffma2_rn(ndG, prev, prev);
    const float2 t = __fadd2_rn(__fadd2_rn(__ffma2_rn(gp, bc2(-1.f), cur), cur), wq);
    return __ffma2_rn(ndG, t, t);
}

__device__ __forceinline__ float4 leapfrog(float4 ndG, float4 cur, float4 prev, float4 T, float4 wh, float4 wl)
{
    return cat2(leap2(lo2(ndG), lo2(cur), lo2(prev), lo2(T), lo2(wh), lo2(wl)),
                leap2(hi2(ndG), hi2(cur), hi2(prev), hi2(T), hi2(wh), hi2(wl)));
}

// a + b
__device__ __forceinline__ float4 add4(float4 a, float4 b)
{
    return cat2(__fadd2_rn(lo2(a), lo2(b)), __fadd2_rn(hi2(a), hi2(b)));
}

// Born scattered source Td - rho T (one rounding per cell)
__device__ __forceinline__ float4 born_src(float4 Td, float4 rho, float4 T)
{
    const float2 m1 = bc2(-1.f);
    return cat2(__ffma2_rn(__fmul2_rn(lo2(rho), m1), lo2(T), lo2(Td)),
                __ffma2_rn(__fmul2_rn(hi2(rho), m1), hi2(T), hi2(Td)));
}

// im + (sc z) Tu: one imaging-condition term
__device__ __forceinline__ float4 image_acc(float4 im, float4 sc, float4 z, float4 Tu)
{
    return cat2(__ffma2_rn(__fmul2_rn(lo2(sc), lo2(z)), lo2(Tu), lo2(im)),
                __ffma2_rn(__fmul2_rn(hi2(sc), hi2(z)), hi2(Tu), hi2(im)));
}

// Add w to the component of q whose cell index is src (pt: index of q.x).
__device__ __forceinline__ void add_source(float4 &q, int src, int pt, float w)
{
    const int d = src - pt;
    if (d >= 0 && d < 4) {
        if (d == 0) q.x = __fadd_rn(q.x, w);
        else if (d == 1) q.y = __fadd_rn(q.y, w);
        else if (d == 2) q.z = __fadd_rn(q.z, w);
        else q.w = __fadd_rn(q.w, w);
    }
}

}  // namespace aafwi
