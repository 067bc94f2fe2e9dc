// reduce_kernels.cu -- FP64-accumulated reductions: the data misfit (eq. FWI)
// and the Anderson-acceleration step (Sec. 2.1 eqs. Ak, solveGamma,
// AA2_update; Sec. 3 Alg. 2).
//
// Every reduction is two-pass with a fixed grid (RED_BLOCKS blocks, grid-
// stride loops, warp-shuffle then shared-memory tree inside a block, the block
// partials summed in block order by the second pass), so results do not depend
// on scheduling.
#include "internal.cuh"
#include "reduce.cuh"

namespace aafwi {

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
// y = a x + b y, then clipped to [lo, hi] when lo < hi
__global__ void __launch_bounds__(RT) k_axpby(float a, const float *x, float b, float *y, long long n, float lo,
                                              float hi)
{
    const bool clip = lo < hi;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        float v = fmaf(a, x[i], b * y[i]);
        if (clip) v = fminf(fmaxf(v, lo), hi);
        y[i] = v;
    }
}

void launch_axpby(float a, const float *x, float b, float *y, long long n, cudaStream_t st, float lo, float hi)
{
    count_launch();
    k_axpby<<<RED_BLOCKS, RT, 0, st>>>(a, x, b, y, n, lo, hi);
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

// The least squares of Alg. 2 step 2 (eqs. Ak, solveGamma) in the gamma
// form: gamma = argmin || dG gamma - G_k ||, dG_j = G_{j+1} - G_j over the
// window.  Its normal matrix and right-hand side are accumulated from the
// differences themselves: dG_j is formed per element in FP64 from the FP32
// ring (exact), so near convergence, when ||dG|| << ||G||, nothing cancels
// (differences of Gram entries of the G_i would lose log10(||G||^2/||dG||^2)
// digits).  The matrix H = dG^T dG is kept by difference across iterations:
// difference j is named by the ring slot of its newer end, and each step adds
// the inner products of the newest difference with all of them.
struct AASlots {
    int slot[AA_MAXM + 1];
    int c;
};

// Copy (p_k, G_k) into ring slot `head` (the newest of the c chronological
// slots) and accumulate per block, w the diagonal weight of a weighted l2
// norm (Sec. 2.1) or null:
//   partials[b][j]           = <dG_new, dG_j>_w   (dG_new = dG_{c-2})
//   partials[b][AA_MAXM + j] = <dG_j, G_k>_w      for j < c - 1.
__global__ void __launch_bounds__(RT) k_aa_append(const float *p_k, const float *g_k, float *ring_p,
                                                  float *ring_g, long long n, int head, AASlots sl,
                                                  const float *w, double *partials)
{
    __shared__ double sh[RT / 32];
    const int nd = sl.c - 1;
    double accH[AA_MAXM], accB[AA_MAXM];
#pragma unroll
    for (int j = 0; j < AA_MAXM; ++j) accH[j] = accB[j] = 0.0;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        const float gv = g_k[i];
        ring_p[(long long)head * n + i] = p_k[i];
        ring_g[(long long)head * n + i] = gv;
        if (nd < 1) continue;
        const double wi = w ? (double)w[i] : 1.0;
        const double gk = (double)gv;
        const double dnew = gk - (double)ring_g[(long long)sl.slot[nd - 1] * n + i];
        double ga = (double)ring_g[(long long)sl.slot[0] * n + i];
#pragma unroll
        for (int j = 0; j < AA_MAXM; ++j) {
            if (j < nd) {
                const double gb = j + 1 == nd ? gk : (double)ring_g[(long long)sl.slot[j + 1] * n + i];
                const double d = gb - ga;
                accH[j] += wi * dnew * d;
                accB[j] += wi * d * gk;
                ga = gb;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < AA_MAXM; ++j) {   // unrolled: the accumulators stay in registers
        if (j < nd) {
            const double h = block_sum(accH[j], sh);
            const double b = block_sum(accB[j], sh);
            if (threadIdx.x == 0) {
                partials[(long long)blockIdx.x * (2 * AA_MAXM) + j] = h;
                partials[(long long)blockIdx.x * (2 * AA_MAXM) + AA_MAXM + j] = b;
            }
        }
    }
}

// Finish the new row of H and the right-hand side, then solve the normal
// equations H gamma = dG^T G_k in FP64 by Cholesky H = R^T R; while
// min R_jj < tol * max R_jj drop the oldest column and refactor.
// dgram[(M+1) x (M+1)]: H by the slot naming each difference.
__global__ void k_aa_solve(double *dgram, const double *partials, int nblocks, int M1, AASlots sl, double tol,
                           double *gamma, int *meta)
{
    __shared__ double hrow[AA_MAXM], rhs[AA_MAXM];
    const int Mk = sl.c - 1;
    for (int j = threadIdx.x; j < 2 * Mk; j += blockDim.x) {
        const int col = j < Mk ? j : AA_MAXM + (j - Mk);
        double acc = 0.0;
        for (int b = 0; b < nblocks; ++b) acc += partials[(long long)b * (2 * AA_MAXM) + col];
        if (j < Mk) hrow[j] = acc;
        else rhs[j - Mk] = acc;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    auto key = [&](int j) { return sl.slot[j + 1]; };   // slot naming difference j
    for (int j = 0; j < Mk; ++j) {
        dgram[key(Mk - 1) * M1 + key(j)] = hrow[j];
        dgram[key(j) * M1 + key(Mk - 1)] = hrow[j];
    }
    double H[AA_MAXM][AA_MAXM], R[AA_MAXM][AA_MAXM], b[AA_MAXM], y[AA_MAXM];
    for (int a = 0; a < Mk; ++a) {
        for (int q = 0; q < Mk; ++q) H[a][q] = dgram[key(a) * M1 + key(q)];
        b[a] = rhs[a];
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
// gamma form; beta = 1: Alg. 2 step 3), over the columns kept by the solve;
// per element in FP64 from the FP32 ring, rounded once.
__global__ void __launch_bounds__(RT) k_aa_mix(const float *ring_p, const float *ring_g, long long n,
                                               AASlots sl, double eta, double beta_eta, const double *gamma,
                                               const int *meta, float *p_tilde, float *p_bar)
{
    __shared__ double gsh[AA_MAXM];
    __shared__ int first_sh, mk_sh;
    if (threadIdx.x == 0) {
        mk_sh = meta[0];
        first_sh = meta[1];
    }
    if (threadIdx.x < AA_MAXM) gsh[threadIdx.x] = threadIdx.x < meta[0] ? gamma[threadIdx.x] : 0.0;
    __syncthreads();
    const int first = first_sh, mk = mk_sh;
    const int newest = sl.slot[sl.c - 1];
    auto gb = [&](int s, long long i) {
        return (double)ring_p[(long long)s * n + i] - beta_eta * (double)ring_g[(long long)s * n + i];
    };
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        const double pb = (double)ring_p[(long long)newest * n + i] - eta * (double)ring_g[(long long)newest * n + i];
        double pt = gb(newest, i);
        double prev = gb(sl.slot[first], i);
        for (int a = 0; a < mk; ++a) {
            const double cur = gb(sl.slot[first + a + 1], i);
            pt -= gsh[a] * (cur - prev);
            prev = cur;
        }
        p_bar[i] = (float)pb;
        p_tilde[i] = (float)pt;
    }
}

void launch_aa_step(AAState &s, const float *p_k, const float *g_k, cudaStream_t st)
{
    const int M1 = s.M + 1;
    s.head = s.count == 0 ? 0 : (s.head + 1) % M1;
    s.count = s.count < M1 ? s.count + 1 : M1;
    AASlots sl;
    sl.c = s.count;
    for (int t = 0; t < sl.c; ++t) sl.slot[t] = ((s.head - (sl.c - 1) + t) % M1 + M1) % M1;
    for (int t = 0; t < sl.c; ++t) s.slots[t] = sl.slot[t];
    count_launch(2);
    k_aa_append<<<RED_BLOCKS, RT, 0, st>>>(p_k, g_k, s.ring_p, s.ring_g, s.n, s.head, sl, s.weights, s.partials);
    k_aa_solve<<<1, 64, 0, st>>>(s.gram, s.partials, RED_BLOCKS, M1, sl, 1e-6, s.gamma, s.meta);
}

void launch_aa_mix(AAState &s, float *p_tilde, float *p_bar, cudaStream_t st)
{
    AASlots sl;
    sl.c = s.count;
    for (int t = 0; t < sl.c; ++t) sl.slot[t] = s.slots[t];
    count_launch();
    k_aa_mix<<<RED_BLOCKS, RT, 0, st>>>(s.ring_p, s.ring_g, s.n, sl, s.eta, s.beta * s.eta, s.gamma, s.meta,
                                        p_tilde, p_bar);
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
