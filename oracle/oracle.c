/*
 * oracle.c -- plain FP64 CPU reference for the adjoint-state FWI / LSRTM
 * gradient of "Anderson Acceleration for Seismic Inversion" (Yang, 2020).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only tests/, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the
 * CUDA library.
 *
 * Everything here is the discrete recurrence written out point by point, in
 * the order the definitions state it, with no blocking or fusion:
 *
 *   PDE (Sec. 2.2, eq. FWD):  m u_tt - Lap u = s,  u(0) = u_t(0) = 0, m = 1/c^2.
 *   Discretisation (the paper is silent; reading used throughout):
 *     leap-frog in time, 8th-order central Laplacian in space, zero outside
 *     the padded grid, Cerjan sponge G of width nb on all four sides, the
 *     physical model edge-replicated into the sponge (extension E), and
 *     W = dt^2 / m:
 *       u^{n+1} = G (2 u^n - G u^{n-1} + W (L u^n + s^n)),  u^0 = u^{-1} = 0
 *     trace sample n = u^{n+1} at the receivers (R in eq. FWI).
 *   Misfit (Sec. 2.2, eq. FWI): J = 1/2 sum (d - g)^2, no dt factor.
 *   Adjoint (Sec. 2.2, eq. FWI_adj): the exact transpose of the recurrence,
 *     written in z = W G a (a = dJ/du^{n+1}):
 *       z^n = G (2 z^{n+1} - G z^{n+2} + W (L z^{n+1} + R^T r^n)),
 *       z^{nt} = z^{nt+1} = 0, run for n = nt-1 .. 0.
 *   Gradient (Sec. 2.2, eq. adj_grad1, discrete form):
 *       dJ/dm_pad = -(1/m) sum_n z^n (L u^n + s^n),  dJ/dm = E^T (dJ/dm_pad).
 *   Born (Sec. 2.2, eq. Born): exact Jacobian of the recurrence in the
 *     direction dm = rho * m0 (rho dimensionless, extended by E):
 *       du^{n+1} = G (2 du^n - G du^{n-1} + W L du^n) - G W rho (L u0^n + s^n)
 *   Born adjoint: z as above with the Born residual, and
 *       img_pad = -sum_n z^n (L u0^n + s^n),  img = E^T img_pad.
 *   Source (Sec. 4.1 names a Ricker wavelet by its centre frequency f; delay
 *     and amplitude are readings): s^n = a w(t_n) / (dx dz) at the source cell,
 *       w(t) = (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2),  tau = t - 1.5/f,
 *       t_n = n dt, a = 1 unless a caller scales it (linearity pins).
 *     The oracle evaluates w itself from (f, dt); it takes no samples from
 *     its callers.
 *
 * Shots are independent; the per-shot loop may run in parallel (OpenMP) but
 * per-shot results are summed afterwards in shot order, so results do not
 * depend on the thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* 8th-order central second-derivative weights (Fornberg), centre then +-1..4. */
static const double FD_C[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0,
                               8.0 / 315.0, -1.0 / 560.0};
static const double SPONGE_A = 0.015;
static const double OG_PI = 3.14159265358979323846;

typedef struct {
    int nz, nx, nb;         /* physical grid and sponge width (cells) */
    double dz, dx, dt;      /* spacing (m) and time step (s) */
    int S;                  /* number of shots */
    const int *src_iz;      /* [S] physical source coordinates */
    const int *src_ix;
    const int *nt;          /* [S] record length of each shot */
    const int *rec_off;     /* [S+1] CSR offsets into rec_iz/rec_ix */
    const int *rec_iz;      /* physical receiver coordinates */
    const int *rec_ix;
    double freq;            /* Ricker centre frequency f (Hz), > 0 */
    double amp;             /* source amplitude a */
} og_geom;

/* ------------------------------------------------------------------ */
/* Building blocks                                                      */
/* ------------------------------------------------------------------ */

/* Ricker wavelet sample w(t) with centre frequency f and delay t0 = 1.5/f. */
static double ricker_at(double f, double t)
{
    const double t0 = 1.5 / f;
    double a = OG_PI * f * (t - t0);
    a = a * a;
    return (1.0 - 2.0 * a) * exp(-a);
}

/* out[n] = w(n dt), n = 0 .. nt-1 (the samples the shot operators inject). */
void og_ricker(double f, double dt, int nt, double *out)
{
    for (int n = 0; n < nt; ++n) out[n] = ricker_at(f, n * dt);
}

/* out = L u on an NZ x NX grid (x fastest), u = 0 outside the grid. */
void og_laplacian(int NZ, int NX, double dz, double dx, const double *u,
                  double *out)
{
    const double iz2 = 1.0 / (dz * dz), ix2 = 1.0 / (dx * dx);
    for (int i = 0; i < NZ; ++i) {
        for (int j = 0; j < NX; ++j) {
            double sz = FD_C[0] * u[(size_t)i * NX + j];
            double sx = FD_C[0] * u[(size_t)i * NX + j];
            for (int k = 1; k <= 4; ++k) {
                double up = (i - k >= 0) ? u[(size_t)(i - k) * NX + j] : 0.0;
                double dn = (i + k < NZ) ? u[(size_t)(i + k) * NX + j] : 0.0;
                double lf = (j - k >= 0) ? u[(size_t)i * NX + j - k] : 0.0;
                double rt = (j + k < NX) ? u[(size_t)i * NX + j + k] : 0.0;
                sz += FD_C[k] * (up + dn);
                sx += FD_C[k] * (lf + rt);
            }
            out[(size_t)i * NX + j] = sz * iz2 + sx * ix2;
        }
    }
}

/* Distance (cells) of padded index i into the sponge of an axis of length
 * n_pad with sponge width nb: 0 in the interior, nb at the outermost cell. */
static int sponge_depth(int i, int n_pad, int nb)
{
    if (i < nb) return nb - i;
    if (i > n_pad - 1 - nb) return i - (n_pad - 1 - nb);
    return 0;
}

/* Cerjan damping per padded cell: G = g(d_z) g(d_x), g(d) = exp(-(a d)^2). */
void og_sponge(int nz, int nx, int nb, double *G)
{
    const int NZ = nz + 2 * nb, NX = nx + 2 * nb;
    for (int i = 0; i < NZ; ++i) {
        double az = SPONGE_A * sponge_depth(i, NZ, nb);
        for (int j = 0; j < NX; ++j) {
            double ax = SPONGE_A * sponge_depth(j, NX, nb);
            G[(size_t)i * NX + j] = exp(-az * az) * exp(-ax * ax);
        }
    }
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Extension E: padded cell takes the value of the nearest physical cell. */
void og_extend(int nz, int nx, int nb, const double *phys, double *pad)
{
    const int NZ = nz + 2 * nb, NX = nx + 2 * nb;
    for (int i = 0; i < NZ; ++i)
        for (int j = 0; j < NX; ++j)
            pad[(size_t)i * NX + j] =
                phys[(size_t)clampi(i - nb, 0, nz - 1) * nx + clampi(j - nb, 0, nx - 1)];
}

/* E^T: every padded cell is added into the physical cell it replicates. */
void og_extend_adjoint(int nz, int nx, int nb, const double *pad, double *phys)
{
    const int NZ = nz + 2 * nb, NX = nx + 2 * nb;
    memset(phys, 0, sizeof(double) * (size_t)nz * nx);
    for (int i = 0; i < NZ; ++i)
        for (int j = 0; j < NX; ++j)
            phys[(size_t)clampi(i - nb, 0, nz - 1) * nx + clampi(j - nb, 0, nx - 1)] +=
                pad[(size_t)i * NX + j];
}

/* ------------------------------------------------------------------ */
/* General propagator on the padded grid (used by the dot-product pins) */
/* ------------------------------------------------------------------ */

/*
 * Forward recurrence with an arbitrary source field s[n][NZ*NX] (already in
 * the "L u + s" units, i.e. per unit area), recording traces[n][j] = u^{n+1}
 * at padded receiver cells.  W and G are per padded cell.
 */
void og_propagate(int NZ, int NX, double dz, double dx, const double *W,
                  const double *G, int nt, const double *s, int nrec,
                  const int *riz, const int *rix, double *traces)
{
    const size_t N = (size_t)NZ * NX;
    double *um = calloc(N, sizeof(double));   /* u^{n-1} */
    double *u0 = calloc(N, sizeof(double));   /* u^n */
    double *up = calloc(N, sizeof(double));   /* u^{n+1} */
    double *lap = malloc(N * sizeof(double));
    for (int n = 0; n < nt; ++n) {
        og_laplacian(NZ, NX, dz, dx, u0, lap);
        for (size_t p = 0; p < N; ++p)
            up[p] = G[p] * (2.0 * u0[p] - G[p] * um[p] + W[p] * (lap[p] + s[(size_t)n * N + p]));
        for (int j = 0; j < nrec; ++j)
            traces[(size_t)n * nrec + j] = up[(size_t)riz[j] * NX + rix[j]];
        double *t = um; um = u0; u0 = up; up = t;
    }
    free(um); free(u0); free(up); free(lap);
}

/*
 * Transpose of og_propagate: given traces r[n][j], returns z[n][NZ*NX] with
 * <traces(s), r> = sum_n <s^n, z^n>  (z^n = W G a^{n+1}).
 */
void og_propagate_adjoint(int NZ, int NX, double dz, double dx, const double *W,
                          const double *G, int nt, const double *r, int nrec,
                          const int *riz, const int *rix, double *z)
{
    const size_t N = (size_t)NZ * NX;
    double *z2 = calloc(N, sizeof(double));   /* z^{n+2} */
    double *z1 = calloc(N, sizeof(double));   /* z^{n+1} */
    double *rhs = malloc(N * sizeof(double));
    for (int n = nt - 1; n >= 0; --n) {
        og_laplacian(NZ, NX, dz, dx, z1, rhs);
        for (int j = 0; j < nrec; ++j)
            rhs[(size_t)riz[j] * NX + rix[j]] += r[(size_t)n * nrec + j];
        double *zn = z + (size_t)n * N;
        for (size_t p = 0; p < N; ++p)
            zn[p] = G[p] * (2.0 * z1[p] - G[p] * z2[p] + W[p] * rhs[p]);
        memcpy(z2, z1, N * sizeof(double));
        memcpy(z1, zn, N * sizeof(double));
    }
    free(z2); free(z1); free(rhs);
}

/* ------------------------------------------------------------------ */
/* Shot-level operators                                                 */
/* ------------------------------------------------------------------ */

typedef struct {
    int NZ, NX;
    size_t N;
    double *m, *W, *G;   /* padded model, dt^2/m, sponge */
} og_medium;

static void medium_build(const og_geom *g, const double *m_phys, og_medium *md)
{
    md->NZ = g->nz + 2 * g->nb;
    md->NX = g->nx + 2 * g->nb;
    md->N = (size_t)md->NZ * md->NX;
    md->m = malloc(md->N * sizeof(double));
    md->W = malloc(md->N * sizeof(double));
    md->G = malloc(md->N * sizeof(double));
    og_extend(g->nz, g->nx, g->nb, m_phys, md->m);
    og_sponge(g->nz, g->nx, g->nb, md->G);
    for (size_t p = 0; p < md->N; ++p) md->W[p] = g->dt * g->dt / md->m[p];
}

static void medium_free(og_medium *md) { free(md->m); free(md->W); free(md->G); }

static size_t trace_offset(const og_geom *g, int s)
{
    size_t off = 0;
    for (int q = 0; q < s; ++q) off += (size_t)g->nt[q] * (g->rec_off[q + 1] - g->rec_off[q]);
    return off;
}

size_t og_trace_count(const og_geom *g) { return trace_offset(g, g->S); }

/*
 * One shot of the forward recurrence.  If lap_hist != NULL it receives
 * (L u^n + s^n) for n = 0..nt-1, the quantity the imaging conditions use.
 * If du_traces != NULL the Born field (direction rho_pad) is stepped along
 * with u and its receiver samples are written there.
 */
static void shot_forward(const og_geom *g, const og_medium *md, int s,
                         const double *rho_pad, double *traces,
                         double *du_traces, double *lap_hist)
{
    const int NZ = md->NZ, NX = md->NX;
    const size_t N = md->N;
    const int nt = g->nt[s];
    const int nr = g->rec_off[s + 1] - g->rec_off[s];
    const int *riz = g->rec_iz + g->rec_off[s], *rix = g->rec_ix + g->rec_off[s];
    const size_t src = (size_t)(g->src_iz[s] + g->nb) * NX + (g->src_ix[s] + g->nb);
    const double inv_cell = 1.0 / (g->dx * g->dz);
    double *um = calloc(N, sizeof(double)), *u0 = calloc(N, sizeof(double));
    double *up = calloc(N, sizeof(double)), *q = malloc(N * sizeof(double));
    double *dm = NULL, *d0 = NULL, *dp = NULL, *dq = NULL;
    if (du_traces) {
        dm = calloc(N, sizeof(double)); d0 = calloc(N, sizeof(double));
        dp = calloc(N, sizeof(double)); dq = malloc(N * sizeof(double));
    }
    for (int n = 0; n < nt; ++n) {
        /* q = L u^n + s^n */
        og_laplacian(NZ, NX, g->dz, g->dx, u0, q);
        q[src] += g->amp * ricker_at(g->freq, n * g->dt) * inv_cell;
        if (lap_hist) memcpy(lap_hist + (size_t)n * N, q, N * sizeof(double));
        for (size_t p = 0; p < N; ++p)
            up[p] = md->G[p] * (2.0 * u0[p] - md->G[p] * um[p] + md->W[p] * q[p]);
        if (du_traces) {
            og_laplacian(NZ, NX, g->dz, g->dx, d0, dq);
            for (size_t p = 0; p < N; ++p)
                dp[p] = md->G[p] * (2.0 * d0[p] - md->G[p] * dm[p] + md->W[p] * dq[p])
                        - md->G[p] * md->W[p] * rho_pad[p] * q[p];
        }
        for (int j = 0; j < nr; ++j) {
            size_t p = (size_t)(riz[j] + g->nb) * NX + (rix[j] + g->nb);
            if (traces) traces[(size_t)n * nr + j] = up[p];
            if (du_traces) du_traces[(size_t)n * nr + j] = dp[p];
        }
        double *t = um; um = u0; u0 = up; up = t;
        if (du_traces) { t = dm; dm = d0; d0 = dp; dp = t; }
    }
    free(um); free(u0); free(up); free(q);
    if (du_traces) { free(dm); free(d0); free(dp); free(dq); }
}

/*
 * One shot of the adjoint recurrence with residual traces r[n][j]; the image
 * img_pad += scale_p * sum_n z^n (lap_hist^n), scale_p per padded cell.
 */
static void shot_adjoint_image(const og_geom *g, const og_medium *md, int s,
                               const double *r, const double *lap_hist,
                               const double *scale, double *img_pad)
{
    const int NZ = md->NZ, NX = md->NX;
    const size_t N = md->N;
    const int nt = g->nt[s];
    const int nr = g->rec_off[s + 1] - g->rec_off[s];
    const int *riz = g->rec_iz + g->rec_off[s], *rix = g->rec_ix + g->rec_off[s];
    double *z2 = calloc(N, sizeof(double)), *z1 = calloc(N, sizeof(double));
    double *zn = malloc(N * sizeof(double)), *rhs = malloc(N * sizeof(double));
    for (int n = nt - 1; n >= 0; --n) {
        og_laplacian(NZ, NX, g->dz, g->dx, z1, rhs);
        for (int j = 0; j < nr; ++j)
            rhs[(size_t)(riz[j] + g->nb) * NX + (rix[j] + g->nb)] += r[(size_t)n * nr + j];
        for (size_t p = 0; p < N; ++p)
            zn[p] = md->G[p] * (2.0 * z1[p] - md->G[p] * z2[p] + md->W[p] * rhs[p]);
        const double *ln = lap_hist + (size_t)n * N;
        for (size_t p = 0; p < N; ++p) img_pad[p] += scale[p] * zn[p] * ln[p];
        double *t = z2; z2 = z1; z1 = zn; zn = t;
    }
    free(z2); free(z1); free(zn); free(rhs);
}

/* F: m_phys -> traces (CSR: shot s at trace offset, time-major [nt_s][nrec_s]). */
void og_forward(const og_geom *g, const double *m_phys, double *traces)
{
    og_medium md;
    medium_build(g, m_phys, &md);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < g->S; ++s)
        shot_forward(g, &md, s, NULL, traces + trace_offset(g, s), NULL, NULL);
    medium_free(&md);
}

/*
 * FWI gradient: returns J = 1/2 ||F(m) - d_obs||^2 and grad = dJ/dm (physical
 * grid).  resid (optional) receives F(m) - d_obs.
 */
double og_fwi_gradient(const og_geom *g, const double *m_phys, const double *d_obs,
                       double *grad, double *resid)
{
    og_medium md;
    medium_build(g, m_phys, &md);
    const size_t N = md.N;
    double *img = calloc((size_t)g->S * N, sizeof(double));
    double *Js = calloc((size_t)g->S, sizeof(double));
    double *scale = malloc(N * sizeof(double));
    for (size_t p = 0; p < N; ++p) scale[p] = -1.0 / md.m[p];
    #pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < g->S; ++s) {
        const int nt = g->nt[s];
        const int nr = g->rec_off[s + 1] - g->rec_off[s];
        const size_t off = trace_offset(g, s), cnt = (size_t)nt * nr;
        double *tr = malloc(cnt * sizeof(double) + 1);
        double *lh = malloc((size_t)nt * N * sizeof(double));
        shot_forward(g, &md, s, NULL, tr, NULL, lh);
        double J = 0.0;
        for (size_t i = 0; i < cnt; ++i) {
            tr[i] -= d_obs[off + i];
            J += 0.5 * tr[i] * tr[i];
            if (resid) resid[off + i] = tr[i];
        }
        Js[s] = J;
        shot_adjoint_image(g, &md, s, tr, lh, scale, img + (size_t)s * N);
        free(tr); free(lh);
    }
    double J = 0.0;
    double *sum = calloc(N, sizeof(double));
    for (int s = 0; s < g->S; ++s) {
        J += Js[s];
        for (size_t p = 0; p < N; ++p) sum[p] += img[(size_t)s * N + p];
    }
    og_extend_adjoint(g->nz, g->nx, g->nb, sum, grad);
    free(sum); free(img); free(Js); free(scale);
    medium_free(&md);
    return J;
}

/* Born modelling L: rho_phys -> scattered traces at background m0_phys. */
void og_born_forward(const og_geom *g, const double *m0_phys, const double *rho_phys,
                     double *traces)
{
    og_medium md;
    medium_build(g, m0_phys, &md);
    double *rho = malloc(md.N * sizeof(double));
    og_extend(g->nz, g->nx, g->nb, rho_phys, rho);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < g->S; ++s)
        shot_forward(g, &md, s, rho, NULL, traces + trace_offset(g, s), NULL);
    free(rho);
    medium_free(&md);
}

/* Born adjoint L^T: residual traces -> image on the physical grid. */
void og_born_adjoint(const og_geom *g, const double *m0_phys, const double *resid,
                     double *img_phys)
{
    og_medium md;
    medium_build(g, m0_phys, &md);
    const size_t N = md.N;
    double *img = calloc((size_t)g->S * N, sizeof(double));
    double *scale = malloc(N * sizeof(double));
    for (size_t p = 0; p < N; ++p) scale[p] = -1.0;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < g->S; ++s) {
        double *lh = malloc((size_t)g->nt[s] * N * sizeof(double));
        shot_forward(g, &md, s, NULL, NULL, NULL, lh);
        shot_adjoint_image(g, &md, s, resid + trace_offset(g, s), lh, scale,
                           img + (size_t)s * N);
        free(lh);
    }
    double *sum = calloc(N, sizeof(double));
    for (int s = 0; s < g->S; ++s)
        for (size_t p = 0; p < N; ++p) sum[p] += img[(size_t)s * N + p];
    og_extend_adjoint(g->nz, g->nx, g->nb, sum, img_phys);
    free(sum); free(img); free(scale);
    medium_free(&md);
}

int og_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
