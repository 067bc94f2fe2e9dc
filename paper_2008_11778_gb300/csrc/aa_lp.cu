// aa_lp.cu -- Anderson acceleration with the l1 or l-infinity norm in the
// optimisation step (Sec. 2.1: the norm of eq. AAopt may be l1, l2 or
// l-infinity; the first and the last need linear programming).
//
//   gamma = argmin || dG gamma - G_k ||_p,  p = 1 or infinity,
//   dG = [G_{i+1} - G_i] over the columns the l2 rank safeguard keeps.
//
// The n rows never leave the GPU.  Each round makes one pass over the ring
// (dG formed per element in FP64 from the FP32 gradients, as in the l2 path)
// and the host solves a linear programme in the M+1 unknowns (gamma, t):
//   l-infinity: exact working-set method.  min t s.t. |dG_i gamma - G_k,i| <= t
//     over a working set of rows; the pass returns max_i |r_i| and the rows
//     above a threshold; when no row exceeds t the working-set optimum is the
//     optimum over all rows.
//   l1: cutting planes on phi(gamma) = sum_i |r_i|, a convex piecewise-linear
//     function: each pass returns phi and a subgradient dG^T sign(r); the LP
//     minimises the maximum of the cuts; it stops when the best phi found and
//     the LP's lower bound agree to a relative gap.
// Both LPs carry a box |gamma_j| <= B around the l2 solution, which bounds
// them from the first round (B is wide enough that it is never active at
// the solution; the step reports it if it is).
//
// aafwi_lp_min is the host LP solver: the revised simplex method applied to
// the dual of min c^T x s.t. A x <= b (few unknowns, many rows), with the
// previous basis reused when rows are added.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/aafwi.h"
#include "internal.cuh"
#include "reduce.cuh"

using namespace aafwi;

namespace {

// ---------------------------------------------------------------------------
// dense LP: min c^T x  s.t.  A x <= b   (x free, nv unknowns, m rows)
//
// Solved through its dual in standard form,
//   min b^T y  s.t.  A^T y = -c,  y >= 0       (nv equations, m columns),
// whose simplex multipliers pi = B^{-T} b_B are the primal x.  Phase I adds
// one artificial column per equation; Bland's rule (smallest index enters,
// smallest basic index leaves among ties) guarantees termination under
// degeneracy, which cutting-plane LPs have in abundance.
// ---------------------------------------------------------------------------
struct DualSimplex {
    int nv = 0, m = 0;
    std::vector<double> A, b, c;      // A row-major [m][nv]
    std::vector<int> basis;           // nv basic column indices (>= m: artificial nv + (j - m))
    std::vector<double> Binv;         // [nv][nv]
    std::vector<double> xB;           // basic values
    double tol = 1e-11;

    double col(int j, int r) const   // entry r of column j of [A^T | diag(s)]
    {
        if (j < m) return A[(size_t)j * nv + r];
        return j - m == r ? (-c[r] >= 0.0 ? 1.0 : -1.0) : 0.0;
    }

    bool invert()
    {
        std::vector<double> Bm((size_t)nv * nv), I((size_t)nv * nv, 0.0);
        for (int r = 0; r < nv; ++r)
            for (int k = 0; k < nv; ++k) Bm[(size_t)r * nv + k] = col(basis[k], r);
        for (int r = 0; r < nv; ++r) I[(size_t)r * nv + r] = 1.0;
        for (int k = 0; k < nv; ++k) {   // Gauss-Jordan with partial pivoting
            int piv = k;
            for (int r = k + 1; r < nv; ++r)
                if (std::fabs(Bm[(size_t)r * nv + k]) > std::fabs(Bm[(size_t)piv * nv + k])) piv = r;
            if (std::fabs(Bm[(size_t)piv * nv + k]) < 1e-300) return false;
            if (piv != k)
                for (int q = 0; q < nv; ++q) {
                    std::swap(Bm[(size_t)k * nv + q], Bm[(size_t)piv * nv + q]);
                    std::swap(I[(size_t)k * nv + q], I[(size_t)piv * nv + q]);
                }
            const double d = Bm[(size_t)k * nv + k];
            for (int q = 0; q < nv; ++q) {
                Bm[(size_t)k * nv + q] /= d;
                I[(size_t)k * nv + q] /= d;
            }
            for (int r = 0; r < nv; ++r) {
                if (r == k) continue;
                const double f = Bm[(size_t)r * nv + k];
                if (f == 0.0) continue;
                for (int q = 0; q < nv; ++q) {
                    Bm[(size_t)r * nv + q] -= f * Bm[(size_t)k * nv + q];
                    I[(size_t)r * nv + q] -= f * I[(size_t)k * nv + q];
                }
            }
        }
        Binv = I;
        xB.assign(nv, 0.0);   // x_B = B^{-1} (-c)
        for (int r = 0; r < nv; ++r)
            for (int q = 0; q < nv; ++q) xB[r] += Binv[(size_t)r * nv + q] * (-c[q]);
        return true;
    }

    // One phase: minimise cost(j) over the columns allowed by `use`.  In
    // phase II (drive_out) an artificial column still basic at level zero
    // leaves as soon as the entering direction would move it.
    // Returns 0 optimal, 1 unbounded, 2 iteration limit, 3 singular basis.
    template <class Cost, class Use>
    int run(Cost cost, Use use, int max_pivots, bool drive_out = false)
    {
        std::vector<double> pi(nv), u(nv);
        const int ncol = m + nv;
        for (int it = 0; it < max_pivots; ++it) {
            // pi = B^{-T} cost_B
            for (int q = 0; q < nv; ++q) {
                double v = 0.0;
                for (int r = 0; r < nv; ++r) v += Binv[(size_t)r * nv + q] * cost(basis[r]);
                pi[q] = v;
            }
            int enter = -1;
            for (int j = 0; j < ncol && enter < 0; ++j) {   // Bland: the first improving column
                if (!use(j) || std::find(basis.begin(), basis.end(), j) != basis.end()) continue;
                double d = cost(j);
                for (int r = 0; r < nv; ++r) d -= pi[r] * col(j, r);
                double scale = std::fabs(cost(j));
                for (int r = 0; r < nv; ++r) scale = std::max(scale, std::fabs(pi[r] * col(j, r)));
                if (d < -tol * std::max(1.0, scale)) enter = j;
            }
            if (enter < 0) return 0;
            for (int r = 0; r < nv; ++r) {
                double v = 0.0;
                for (int q = 0; q < nv; ++q) v += Binv[(size_t)r * nv + q] * col(enter, q);
                u[r] = v;
            }
            int leave = -1;
            double best = 0.0;
            for (int r = 0; r < nv && drive_out; ++r)
                if (basis[r] >= m && std::fabs(u[r]) > tol && (leave < 0 || basis[r] < basis[leave])) leave = r;
            if (leave < 0) {   // ratio test (Bland: the smallest basic index among ties)
                for (int r = 0; r < nv; ++r) {
                    if (u[r] <= tol) continue;
                    const double ratio = std::max(0.0, xB[r]) / u[r];
                    if (leave < 0 || ratio < best - 1e-15 * std::max(1.0, best) ||
                        (std::fabs(ratio - best) <= 1e-15 * std::max(1.0, best) && basis[r] < basis[leave])) {
                        leave = r;
                        best = ratio;
                    }
                }
            }
            if (leave < 0) return 1;
            basis[leave] = enter;
            if (!invert()) return 3;
        }
        return 2;
    }

    // Solve; keeps the basis for a warm start after rows are appended
    // (appended primal rows are new dual columns: the basis stays feasible).
    int solve(std::vector<double> &x, double *obj)
    {
        const int max_pivots = 50 * (nv + m) + 1000;
        bool warm = (int)basis.size() == nv && invert();
        if (warm)
            for (int r = 0; r < nv; ++r) warm = warm && xB[r] >= -1e-9 * (1.0 + std::fabs(xB[r]));
        if (!warm) {   // phase I from the artificial basis
            basis.resize(nv);
            for (int r = 0; r < nv; ++r) basis[r] = m + r;
            if (!invert()) return 3;
            const int rc = run([&](int j) { return j >= m ? 1.0 : 0.0; }, [&](int) { return true; }, max_pivots);
            if (rc) return rc == 1 ? 4 : rc;
            double infeas = 0.0, scale = 1.0;
            for (int r = 0; r < nv; ++r) {
                if (basis[r] >= m) infeas += std::fabs(xB[r]);
                scale = std::max(scale, std::fabs(c[r]));
            }
            if (infeas > 1e-9 * scale) return 5;   // the dual is infeasible: primal unbounded
            // drive zero-level artificials out of the basis where a real column can replace them
            for (int r = 0; r < nv; ++r) {
                if (basis[r] < m) continue;
                for (int j = 0; j < m; ++j) {
                    if (std::find(basis.begin(), basis.end(), j) != basis.end()) continue;
                    double v = 0.0;
                    for (int q = 0; q < nv; ++q) v += Binv[(size_t)r * nv + q] * col(j, q);
                    if (std::fabs(v) > 1e-9) {
                        const int old = basis[r];
                        basis[r] = j;
                        if (invert()) break;
                        basis[r] = old;
                        invert();
                    }
                }
            }
        }
        const int rc = run([&](int j) { return j < m ? b[j] : 0.0; }, [&](int j) { return j < m; }, max_pivots, true);
        if (rc) return rc == 1 ? 5 : rc;
        x.assign(nv, 0.0);
        for (int q = 0; q < nv; ++q) {
            double v = 0.0;
            for (int r = 0; r < nv; ++r) v += Binv[(size_t)r * nv + q] * (basis[r] < m ? b[basis[r]] : 0.0);
            x[q] = v;
        }
        if (obj) {
            double v = 0.0;
            for (int q = 0; q < nv; ++q) v += c[q] * x[q];
            *obj = v;
        }
        return 0;
    }

    void add_row(const double *a, double bi)
    {
        A.insert(A.end(), a, a + nv);
        b.push_back(bi);
        // artificial columns are numbered after the real ones: shift them
        for (int &k : basis)
            if (k >= m) ++k;
        ++m;
    }
};

const char *lp_status_text(int rc)
{
    switch (rc) {
    case 2: return "iteration limit";
    case 3: return "singular basis";
    case 4: return "phase I unbounded";
    case 5: return "unbounded or infeasible";
    default: return "failed";
    }
}

// ---------------------------------------------------------------------------
// kernels: one pass over the ring per round
// ---------------------------------------------------------------------------

struct LpCols {
    int slot[AA_MAXM + 1];   // chronological slots of the kept window: dG_j = G[slot[j+1]] - G[slot[j]]
    int mk;                  // columns
    double gam[AA_MAXM];     // current gamma
};

// r_i = sum_j gamma_j dG_j,i - G_k,i in FP64; per block:
//   l1 (want_sub): partials[b][0] = sum w_i |r_i|, partials[b][1 + j] = sum w_i sign(r_i) dG_j,i
//   l-infinity:    partials[b][0] = max |r_i|;  rows with |r_i| > thr appended to rows[] (count in *cnt)
__global__ void __launch_bounds__(RT) k_lp_pass(const float *ring_g, long long n, LpCols lc, const float *w,
                                               int want_sub, double thr, int *rows, int cap, int *cnt,
                                               double *partials)
{
    __shared__ double sh[RT / 32];
    double acc0 = 0.0, sub[AA_MAXM];
#pragma unroll
    for (int j = 0; j < AA_MAXM; ++j) sub[j] = 0.0;
    const long long newest = lc.slot[lc.mk];
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        const double gk = (double)ring_g[newest * n + i];
        double ga = (double)ring_g[(long long)lc.slot[0] * n + i];
        double d[AA_MAXM];
        double r = -gk;
#pragma unroll
        for (int j = 0; j < AA_MAXM; ++j) {
            d[j] = 0.0;
            if (j < lc.mk) {
                const double gb = (double)ring_g[(long long)lc.slot[j + 1] * n + i];
                d[j] = gb - ga;
                r += lc.gam[j] * d[j];
                ga = gb;
            }
        }
        const double wi = w ? (double)w[i] : 1.0;
        if (want_sub) {
            acc0 += wi * fabs(r);
            const double sg = r > 0.0 ? wi : (r < 0.0 ? -wi : 0.0);
#pragma unroll
            for (int j = 0; j < AA_MAXM; ++j)
                if (j < lc.mk) sub[j] += sg * d[j];
        } else {
            const double a = wi * fabs(r);
            acc0 = fmax(acc0, a);
            if (a > thr) {
                const int k = atomicAdd(cnt, 1);
                if (k < cap) rows[k] = (int)i;
            }
        }
    }
    if (want_sub) {
        const double v = block_sum(acc0, sh);
        if (threadIdx.x == 0) partials[(long long)blockIdx.x * (AA_MAXM + 1)] = v;
#pragma unroll
        for (int j = 0; j < AA_MAXM; ++j) {
            if (j < lc.mk) {
                const double s = block_sum(sub[j], sh);
                if (threadIdx.x == 0) partials[(long long)blockIdx.x * (AA_MAXM + 1) + 1 + j] = s;
            }
        }
    } else {
        const double v = block_max(acc0, sh);
        if (threadIdx.x == 0) partials[(long long)blockIdx.x * (AA_MAXM + 1)] = v;
    }
}

// For each listed row: (dG_0..dG_{mk-1}, G_k, w) of that row, FP64.
__global__ void k_lp_gather(const float *ring_g, long long n, LpCols lc, const float *w, const int *rows, int nr,
                            double *out)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nr) return;
    const long long i = rows[q];
    double *o = out + (long long)q * (AA_MAXM + 2);
    double ga = (double)ring_g[(long long)lc.slot[0] * n + i];
    for (int j = 0; j < lc.mk; ++j) {
        const double gb = (double)ring_g[(long long)lc.slot[j + 1] * n + i];
        o[j] = gb - ga;
        ga = gb;
    }
    o[AA_MAXM] = (double)ring_g[(long long)lc.slot[lc.mk] * n + i];
    o[AA_MAXM + 1] = w ? (double)w[i] : 1.0;
}

struct Pass {
    double v0;                 // l1: phi; l-infinity: max |r|
    std::vector<double> sub;   // l1 subgradient
};

}  // namespace

namespace aafwi {

// gamma of the l1 / l-infinity least-deviation problem over the kept window
// (see the file header); gamma_in: the l2 solution (start and box centre).
// Writes gamma[0..mk) and returns AAFWI_OK, or an error with a message.
int aa_lp_gamma(AAState &s, const int *slots, int mk, int norm, const double *gamma_in, double *gamma,
                AALpStats *stats, std::string *msg, cudaStream_t st)
{
    const long long n = s.n;
    LpCols lc{};
    for (int j = 0; j <= mk; ++j) lc.slot[j] = slots[j];
    lc.mk = mk;
    for (int j = 0; j < mk; ++j) lc.gam[j] = gamma_in[j];
    const int nv = mk + 1;   // gamma, t (l-infinity) or theta (l1)
    double B = 0.0;
    for (int j = 0; j < mk; ++j) B = std::max(B, std::fabs(gamma_in[j]));
    B = 1e3 * std::max(1.0, B);
    DualSimplex lp;
    lp.nv = nv;
    lp.c.assign(nv, 0.0);
    lp.c[mk] = 1.0;   // minimise t / theta
    std::vector<double> row(nv);
    for (int j = 0; j < mk; ++j) {   // box rows
        std::fill(row.begin(), row.end(), 0.0);
        row[j] = 1.0;
        lp.add_row(row.data(), B);
        row[j] = -1.0;
        lp.add_row(row.data(), B);
    }
    std::vector<double> part((size_t)RED_BLOCKS * (AA_MAXM + 1));
    auto pass = [&](bool l1, double thr, int *nrows, Pass *out) -> int {
        if (cudaMemsetAsync(s.lp_cnt, 0, sizeof(int), st) != cudaSuccess) return AAFWI_ERR_CUDA;
        count_launch();
        k_lp_pass<<<RED_BLOCKS, RT, 0, st>>>(s.ring_g, n, lc, s.weights, l1 ? 1 : 0, thr, s.lp_rows,
                                            AA_LP_ROWS, s.lp_cnt, s.lp_part);
        cudaError_t e = cudaMemcpyAsync(part.data(), s.lp_part, part.size() * sizeof(double),
                                        cudaMemcpyDeviceToHost, st);
        int cnt = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, s.lp_cnt, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return AAFWI_ERR_CUDA;
        out->v0 = 0.0;
        out->sub.assign(mk, 0.0);
        for (int b = 0; b < RED_BLOCKS; ++b) {   // fixed order: deterministic
            const double *p = &part[(size_t)b * (AA_MAXM + 1)];
            out->v0 = l1 ? out->v0 + p[0] : std::max(out->v0, p[0]);
            if (l1)
                for (int j = 0; j < mk; ++j) out->sub[j] += p[1 + j];
        }
        if (nrows) *nrows = cnt;
        return AAFWI_OK;
    };
    std::vector<double> x;
    int rounds = 0;
    if (norm == AAFWI_NORM_L1) {
        // cutting planes: theta >= phi(g_r) + sub_r (gamma - g_r)
        double best = -1.0, lower = -1e300, sigma = 0.0;   // cuts in units of phi(gamma_l2)
        std::vector<double> gbest(gamma_in, gamma_in + mk), g(gamma_in, gamma_in + mk);
        for (rounds = 1; rounds <= AA_LP_MAX_ROUNDS; ++rounds) {
            for (int j = 0; j < mk; ++j) lc.gam[j] = g[j];
            Pass P;
            if (pass(true, 0.0, nullptr, &P)) return AAFWI_ERR_CUDA;
            if (rounds == 1) {
                sigma = P.v0;
                if (!(sigma > 0.0)) {   // G_k = dG gamma_l2 exactly: nothing to improve
                    best = lower = 0.0;
                    break;
                }
            }
            if (best < 0.0 || P.v0 < best) {
                best = P.v0;
                gbest = g;
            }
            if (best - lower <= AA_LP_GAP * best) break;
            double rhs = -P.v0 / sigma;
            for (int j = 0; j < mk; ++j) {
                row[j] = P.sub[j] / sigma;
                rhs += row[j] * g[j];
            }
            row[mk] = -1.0;
            lp.add_row(row.data(), rhs);
            double obj = 0.0;
            const int rc = lp.solve(x, &obj);
            if (rc) {
                *msg = std::string("aa_step (l1): LP ") + lp_status_text(rc);
                return AAFWI_ERR_STATE;
            }
            lower = obj * sigma;
            for (int j = 0; j < mk; ++j) g[j] = x[j];
            if (best - lower <= AA_LP_GAP * best) {   // the new point cannot improve by more than the gap
                for (int j = 0; j < mk; ++j) lc.gam[j] = g[j];
                if (pass(true, 0.0, nullptr, &P)) return AAFWI_ERR_CUDA;
                if (P.v0 < best) {
                    best = P.v0;
                    gbest = g;
                }
                break;
            }
        }
        if (rounds > AA_LP_MAX_ROUNDS) {
            *msg = "aa_step (l1): cutting planes did not close the gap within the round limit";
            return AAFWI_ERR_STATE;
        }
        for (int j = 0; j < mk; ++j) gamma[j] = gbest[j];
        if (stats) {
            stats->objective = best;
            stats->lower_bound = lower;
            stats->rounds = rounds;
            stats->rows = lp.m - 2 * mk;
        }
    } else {
        // working set: start from the rows with the largest |G_k,i| (at gamma = 0)
        std::vector<int> rows_h(AA_LP_ROWS);
        std::vector<double> gat((size_t)AA_LP_ROWS * (AA_MAXM + 2));
        std::vector<int> ws;
        for (int j = 0; j < mk; ++j) lc.gam[j] = 0.0;
        Pass P;
        int cnt = 0;
        if (pass(false, 1e300, nullptr, &P)) return AAFWI_ERR_CUDA;   // max w |G_k|
        const double sigma = P.v0;   // rows in units of max w |G_k|
        if (!(sigma > 0.0)) {
            for (int j = 0; j < mk; ++j) gamma[j] = 0.0;
            if (stats) *stats = AALpStats{};
            return AAFWI_OK;
        }
        double tcur = -1.0;   // current LP level: rows above it are violated
        double thr = 0.5 * P.v0;
        for (rounds = 1; rounds <= AA_LP_MAX_ROUNDS; ++rounds) {
            // rows above thr at the current gamma; raise thr until they fit the buffer
            int tries = 0;
            for (;;) {
                if (pass(false, thr, &cnt, &P)) return AAFWI_ERR_CUDA;
                if (cnt <= AA_LP_ROWS || ++tries > 60) break;
                thr = 0.5 * (thr + P.v0);
            }
            if (tcur >= 0.0 && P.v0 <= tcur * (1.0 + AA_LP_GAP)) break;   // no row exceeds the level: optimal
            const int nr = std::min(cnt, AA_LP_ROWS);
            if (cudaMemcpyAsync(rows_h.data(), s.lp_rows, nr * sizeof(int), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess)
                return AAFWI_ERR_CUDA;
            if (cudaStreamSynchronize(st) != cudaSuccess) return AAFWI_ERR_CUDA;
            std::sort(rows_h.begin(), rows_h.begin() + nr);   // deterministic order
            std::vector<int> add;
            for (int q = 0; q < nr; ++q)
                if (!std::binary_search(ws.begin(), ws.end(), rows_h[q])) add.push_back(rows_h[q]);
            if (add.empty()) {
                *msg = "aa_step (l-infinity): no new row above the level";
                return AAFWI_ERR_STATE;
            }
            if (cudaMemcpyAsync(s.lp_rows, add.data(), add.size() * sizeof(int), cudaMemcpyHostToDevice, st) !=
                cudaSuccess)
                return AAFWI_ERR_CUDA;
            count_launch();
            k_lp_gather<<<((int)add.size() + 127) / 128, 128, 0, st>>>(s.ring_g, n, lc, s.weights, s.lp_rows,
                                                                      (int)add.size(), s.lp_gat);
            if (cudaMemcpyAsync(gat.data(), s.lp_gat, add.size() * (AA_MAXM + 2) * sizeof(double),
                                cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return AAFWI_ERR_CUDA;
            for (size_t q = 0; q < add.size(); ++q) {   // w (dG gamma - G_k) <= t and -w (...) <= t
                const double *o = &gat[q * (AA_MAXM + 2)];
                const double wi = o[AA_MAXM + 1] / sigma;
                for (int j = 0; j < mk; ++j) row[j] = wi * o[j];
                row[mk] = -1.0;
                lp.add_row(row.data(), wi * o[AA_MAXM]);
                for (int j = 0; j < mk; ++j) row[j] = -wi * o[j];
                lp.add_row(row.data(), -wi * o[AA_MAXM]);
            }
            ws.insert(ws.end(), add.begin(), add.end());
            std::sort(ws.begin(), ws.end());
            double obj = 0.0;
            const int rc = lp.solve(x, &obj);
            if (rc) {
                *msg = std::string("aa_step (l-infinity): LP ") + lp_status_text(rc);
                return AAFWI_ERR_STATE;
            }
            tcur = obj * sigma;
            for (int j = 0; j < mk; ++j) lc.gam[j] = x[j];
            thr = tcur * (1.0 + AA_LP_GAP);
        }
        if (rounds > AA_LP_MAX_ROUNDS) {
            *msg = "aa_step (l-infinity): working set did not converge within the round limit";
            return AAFWI_ERR_STATE;
        }
        for (int j = 0; j < mk; ++j) gamma[j] = lc.gam[j];
        if (stats) {
            stats->objective = P.v0;
            stats->lower_bound = tcur;
            stats->rounds = rounds;
            stats->rows = (int)ws.size();
        }
    }
    bool box = false;
    for (int j = 0; j < mk; ++j) box = box || std::fabs(gamma[j]) >= B * (1.0 - 1e-9);
    if (box) {
        *msg = "aa_step: the l1 / l-infinity solution reached the box around the l2 solution";
        return AAFWI_ERR_STATE;
    }
    return AAFWI_OK;
}

}  // namespace aafwi

extern "C" int aafwi_lp_min(int nv, int m, const double *A, const double *b, const double *c, double *x,
                            double *obj)
{
    if (nv < 1 || nv > 64 || m < 0 || (m > 0 && (!A || !b)) || !c || !x) {
        set_call_error("lp_min: invalid argument");
        return AAFWI_ERR_ARG;
    }
    DualSimplex lp;
    lp.nv = nv;
    lp.c.assign(c, c + nv);
    for (int i = 0; i < m; ++i) lp.add_row(A + (size_t)i * nv, b[i]);
    std::vector<double> xs;
    const int rc = lp.solve(xs, obj);
    if (rc) {
        set_call_error(std::string("lp_min: ") + lp_status_text(rc));
        return AAFWI_ERR_STATE;
    }
    std::copy(xs.begin(), xs.end(), x);
    return AAFWI_OK;
}
