// reduce_kernels.cu -- FP64-accumulated reductions: the data misfit (eq. FWI)
// and the Anderson-acceleration step (Sec. 2.1 eqs. Ak, solveGamma,
// AA2_update; Sec. 3 Alg. 2).
//
// Every reduction is two-pass with a fixed grid (RED_BLOCKS blocks, grid-
// stride loops, warp-shuffle then shared-memory tree inside a block, the block
// partials summed in block order by the second pass), so results do not depend
// on scheduling.
#include "internal.cuh"

namespace aafwi {

constexpr int RT = 256;  // threads per reduction block

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    v = threadIdx.x < RT / 32 ? sh[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    return v;
}

__global__ void __launch_bounds__(RT) k_misfit(const float *d, const float *o, float *r, long long n,
                                               double *partials)
{
    __shared__ double sh[RT / 32];
    double acc = 0.0;
    const long long n4 = n / 4;
    const bool vec = ((reinterpret_cast<uintptr_t>(d) | reinterpret_cast<uintptr_t>(o) |
                       reinterpret_cast<uintptr_t>(r)) & 15) == 0;
    const long long stride = (long long)gridDim.x * RT;
    long long i0 = 0;
    if (vec) {
        for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n4; i += stride) {
            const float4 a = reinterpret_cast<const float4 *>(d)[i];
            const float4 b = reinterpret_cast<const float4 *>(o)[i];
            const float4 e = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
            if (r) reinterpret_cast<float4 *>(r)[i] = e;
            acc += (double)e.x * e.x + (double)e.y * e.y + (double)e.z * e.z + (double)e.w * e.w;
        }
        i0 = n4 * 4;
    }
    for (long long i = i0 + blockIdx.x * (long long)RT + threadIdx.x; i < n; i += stride) {
        const float e = d[i] - o[i];
        if (r) r[i] = e;
        acc += (double)e * e;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// out = scale * sum of nb partials (fixed order per thread, then tree).
__global__ void __launch_bounds__(RT) k_finish_sum(const double *partials, int nb, double scale,
                                                   double *out)
{
    __shared__ double sh[RT / 32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += RT) acc += partials[i];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) *out = scale * acc;
}

void launch_misfit(const float *d_syn, const float *d_obs, float *resid, long long n,
                   double *partials, double *J_dev, cudaStream_t st)
{
    count_launch(2);
    k_misfit<<<RED_BLOCKS, RT, 0, st>>>(d_syn, d_obs, resid, n, partials);
    k_finish_sum<<<1, RT, 0, st>>>(partials, RED_BLOCKS, 0.5, J_dev);
}

// <x, y> accumulated in FP64: block partials (grid-stride, fixed grid).
__global__ void __launch_bounds__(RT) k_dot(const float *x, const float *y, long long n, double *partials)
{
    __shared__ double sh[RT / 32];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT)
        acc += (double)x[i] * (double)y[i];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

void launch_dot(const float *x, const float *y, long long n, double *partials, double *out_dev, cudaStream_t st)
{
    count_launch(2);
    k_dot<<<RED_BLOCKS, RT, 0, st>>>(x, y, n, partials);
    k_finish_sum<<<1, RT, 0, st>>>(partials, RED_BLOCKS, 1.0, out_dev);
}

// y = a x + b y
__global__ void __launch_bounds__(RT) k_axpby(float a, const float *x, float b, float *y, long long n)
{
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT)
        y[i] = fmaf(a, x[i], b * y[i]);
}

void launch_axpby(float a, const float *x, float b, float *y, long long n, cudaStream_t st)
{
    count_launch();
    k_axpby<<<RED_BLOCKS, RT, 0, st>>>(a, x, b, y, n);
}

__global__ void __launch_bounds__(RT) k_absmax(const float *x, long long n, double *partials)
{
    __shared__ double sh[RT / 32];
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT)
        m = fmax(m, fabs((double)x[i]));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < RT / 32 ? sh[threadIdx.x] : 0.0;
        m = warp_max(m);
        if (threadIdx.x == 0) partials[blockIdx.x] = m;
    }
}

__global__ void k_finish_max(const double *partials, int nb, double *out)
{
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < nb; ++i) m = fmax(m, partials[i]);
        *out = m;
    }
}

void launch_absmax(const float *x, long long n, double *partials, double *out_dev, cudaStream_t st)
{
    count_launch(2);
    k_absmax<<<RED_BLOCKS, RT, 0, st>>>(x, n, partials);
    k_finish_max<<<1, 32, 0, st>>>(partials, RED_BLOCKS, out_dev);
}

// ---------------------------------------------------------------------------
// Anderson acceleration
// ---------------------------------------------------------------------------

// Copy (p_k, G_k) into ring slot `head` and accumulate <G_k, G_slot>_w for the
// c history slots (chronological slot list `slots`, the newest last); w: the
// diagonal weight of a weighted l2 norm (Sec. 2.1), or null for the l2 norm.
struct AASlots {
    int slot[AA_MAXM + 1];
    int c;
};

__global__ void __launch_bounds__(RT) k_aa_append(const float *p_k, const float *g_k, float *ring_p,
                                                  float *ring_g, long long n, int head, AASlots sl,
                                                  const float *w, double *partials)
{
    __shared__ double sh[RT / 32];
    double acc[AA_MAXM + 1];
#pragma unroll
    for (int j = 0; j <= AA_MAXM; ++j) acc[j] = 0.0;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        const float gv = g_k[i];
        ring_p[(long long)head * n + i] = p_k[i];
        ring_g[(long long)head * n + i] = gv;
        const double gw = w ? (double)w[i] * (double)gv : (double)gv;
#pragma unroll
        for (int j = 0; j <= AA_MAXM; ++j) {
            if (j < sl.c) {
                const float o = sl.slot[j] == head ? gv : ring_g[(long long)sl.slot[j] * n + i];
                acc[j] += gw * (double)o;
            }
        }
    }
    for (int j = 0; j < sl.c; ++j) {
        const double v = block_sum(acc[j], sh);
        if (threadIdx.x == 0) partials[(long long)blockIdx.x * (AA_MAXM + 2) + j] = v;
    }
}

// Finish the new Gram row, then solve the small least-squares problem
// gamma = argmin || dG gamma - G_k || through the normal equations in FP64:
// H = dG^T dG from the Gram matrix of the history gradients, Cholesky
// H = R^T R; while min R_jj < tol * max R_jj drop the oldest column.
__global__ void k_aa_solve(double *gram, const double *partials, int nblocks, int M1, int head,
                           AASlots sl, double tol, double *gamma, int *meta)
{
    __shared__ double row[AA_MAXM + 1];
    const int c = sl.c;
    for (int j = threadIdx.x; j < c; j += blockDim.x) {
        double acc = 0.0;
        for (int b = 0; b < nblocks; ++b) acc += partials[(long long)b * (AA_MAXM + 2) + j];
        row[j] = acc;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int j = 0; j < c; ++j) {
        gram[head * M1 + sl.slot[j]] = row[j];
        gram[sl.slot[j] * M1 + head] = row[j];
    }
    const int Mk = c - 1;
    double H[AA_MAXM][AA_MAXM], R[AA_MAXM][AA_MAXM], b[AA_MAXM], y[AA_MAXM];
    auto G = [&](int a, int bb) { return gram[sl.slot[a] * M1 + sl.slot[bb]]; };
    for (int a = 0; a < Mk; ++a) {
        for (int q = 0; q < Mk; ++q)
            H[a][q] = G(a + 1, q + 1) - G(a + 1, q) - G(a, q + 1) + G(a, q);
        b[a] = G(a + 1, Mk) - G(a, Mk);
    }
    int first = 0;
    for (; first < Mk; ++first) {
        const int m = Mk - first;
        bool ok = true;
        double dmin = 1e300, dmax = 0.0;
        for (int j = 0; j < m && ok; ++j) {
            double d = H[first + j][first + j];
            for (int k = 0; k < j; ++k) d -= R[k][j] * R[k][j];
            if (!(d > 0.0)) { ok = false; break; }
            R[j][j] = sqrt(d);
            for (int i = j + 1; i < m; ++i) {
                double v = H[first + j][first + i];
                for (int k = 0; k < j; ++k) v -= R[k][j] * R[k][i];
                R[j][i] = v / R[j][j];
            }
            dmin = fmin(dmin, R[j][j]);
            dmax = fmax(dmax, R[j][j]);
        }
        if (ok && dmin >= tol * dmax) {
            // R^T y = b, then R gamma = y
            for (int j = 0; j < m; ++j) {
                double v = b[first + j];
                for (int k = 0; k < j; ++k) v -= R[k][j] * y[k];
                y[j] = v / R[j][j];
            }
            for (int j = m - 1; j >= 0; --j) {
                double v = y[j];
                for (int k = j + 1; k < m; ++k) v -= R[j][k] * gamma[k];
                gamma[j] = v / R[j][j];
            }
            break;
        }
    }
    meta[0] = Mk - first;
    meta[1] = first;
}

// p_bar = p_k - eta G_k;  p_tilde = Gb_k - sum_a gamma_a (Gb_{a+1} - Gb_a),
// Gb_i = p_i - beta eta G_i (the damped update of Alg. 1 eq. AAupdate0 in the
// gamma form; beta = 1: Alg. 2 step 3), over the columns kept by the solve.
__global__ void __launch_bounds__(RT) k_aa_mix(const float *ring_p, const float *ring_g, long long n,
                                               AASlots sl, float eta, float beta_eta, const double *gamma,
                                               const int *meta, float *p_tilde, float *p_bar)
{
    __shared__ float gsh[AA_MAXM];
    __shared__ int first_sh, mk_sh;
    if (threadIdx.x == 0) {
        mk_sh = meta[0];
        first_sh = meta[1];
    }
    if (threadIdx.x < AA_MAXM) gsh[threadIdx.x] = threadIdx.x < meta[0] ? (float)gamma[threadIdx.x] : 0.f;
    __syncthreads();
    const int first = first_sh, mk = mk_sh;
    const int newest = sl.slot[sl.c - 1];
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        const float pb = ring_p[(long long)newest * n + i] - eta * ring_g[(long long)newest * n + i];
        float pt = ring_p[(long long)newest * n + i] - beta_eta * ring_g[(long long)newest * n + i];
        float prev = ring_p[(long long)sl.slot[first] * n + i] - beta_eta * ring_g[(long long)sl.slot[first] * n + i];
        for (int a = 0; a < mk; ++a) {
            const int sn = sl.slot[first + a + 1];
            const float cur = ring_p[(long long)sn * n + i] - beta_eta * ring_g[(long long)sn * n + i];
            pt -= gsh[a] * (cur - prev);
            prev = cur;
        }
        p_bar[i] = pb;
        p_tilde[i] = pt;
    }
}

void launch_aa_step(AAState &s, const float *p_k, const float *g_k, float *p_tilde, float *p_bar,
                    cudaStream_t st)
{
    const int M1 = s.M + 1;
    s.head = s.count == 0 ? 0 : (s.head + 1) % M1;
    s.count = s.count < M1 ? s.count + 1 : M1;
    AASlots sl;
    sl.c = s.count;
    for (int t = 0; t < sl.c; ++t) sl.slot[t] = ((s.head - (sl.c - 1) + t) % M1 + M1) % M1;
    count_launch(3);
    k_aa_append<<<RED_BLOCKS, RT, 0, st>>>(p_k, g_k, s.ring_p, s.ring_g, s.n, s.head, sl, s.weights, s.partials);
    k_aa_solve<<<1, 32, 0, st>>>(s.gram, s.partials, RED_BLOCKS, M1, s.head, sl, 1e-6, s.gamma, s.meta);
    k_aa_mix<<<RED_BLOCKS, RT, 0, st>>>(s.ring_p, s.ring_g, s.n, sl, (float)s.eta, (float)(s.beta * s.eta),
                                        s.gamma, s.meta, p_tilde, p_bar);
}

// p_next = clip(lam p_tilde + (1 - lam) p_bar); partial <G_k, p_next - p_k>.
__global__ void __launch_bounds__(RT) k_aa_combine(const float *p_tilde, const float *p_bar, float *p_next,
                                                   long long n, float lam, float lo, float hi,
                                                   const float *p_k, const float *g_k, double *partials)
{
    __shared__ double sh[RT / 32];
    double acc = 0.0;
    const bool clip = lo < hi;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        float v = lam * p_tilde[i] + (1.f - lam) * p_bar[i];
        if (clip) v = fminf(fmaxf(v, lo), hi);
        p_next[i] = v;
        if (partials) acc += (double)g_k[i] * ((double)v - (double)p_k[i]);
    }
    if (partials) {
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) partials[blockIdx.x] = acc;
    }
}

void launch_aa_combine(AAState &s, float lam, const float *p_tilde, const float *p_bar, float *p_next,
                       float lo, float hi, bool want_dot, cudaStream_t st)
{
    const float *pk = s.ring_p + (long long)s.head * s.n;
    const float *gk = s.ring_g + (long long)s.head * s.n;
    count_launch(want_dot ? 2 : 1);
    k_aa_combine<<<RED_BLOCKS, RT, 0, st>>>(p_tilde, p_bar, p_next, s.n, lam, lo, hi, pk, gk,
                                            want_dot ? s.partials : nullptr);
    if (want_dot) k_finish_sum<<<1, RT, 0, st>>>(s.partials, RED_BLOCKS, 1.0, s.dot);
}

}  // namespace aafwi
