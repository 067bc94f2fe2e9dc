// internal.cuh -- kernel argument blocks and launchers shared by the CUDA
// translation units of libaafwi.so.  Not part of the public ABI (aafwi.h).
#pragma once
#include <cuda.h>              // CUtensorMap (TMA descriptors)
#include <cuda_runtime.h>
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/aafwi.h"

namespace aafwi {

// Tile of one CTA of the per-step kernels: tz rows x TX columns of one shot,
// 256 threads laid out 32 (x) x 8 (z); a thread owns 4 consecutive columns
// (one float4) on tz/8 rows (the forward: adjacent rows; the others: rows
// 8 apart).  tz is a plan parameter (16, 32 or 64; the
// kernels are instantiated for each).  HALO = stencil radius of the
// 8th-order Laplacian.
constexpr int HALO = 4;
constexpr int TX = 128;
constexpr int TZ_DEFAULT = 16;
constexpr int BX = 32;
constexpr int BY = 8;
constexpr int SW = TX + 2 * HALO;      // shared tile row length (floats)
constexpr int SW8 = TX + 4 * HALO;     // the same with an 8-cell halo (two-step forward)
inline bool tile_z_supported(int tz) { return tz == 16 || tz == 32 || tz == 64; }

// The per-step kernels stage their inputs with TMA copies from 4D tensor
// maps of the field buffers: (x < NX, z < NZ, shot, slot) with row pitch
// `pitch`.  The box is a tile with a halo of `halo` cells on every side:
// 0 (interior map, tz x TX), HALO (tz + 8 rows x SW columns) or 2 HALO (the
// two-step forward's u^n, tz + 16 rows x SW8 columns); cells outside the
// padded grid (negative or beyond NX / NZ) arrive as zeros.
bool encode_tile_map(CUtensorMap *m, const float *base, int NX, int NZ, int pitch, long long field, int S,
                     int slots, int tile_rows, int halo, std::string *why);

// Per-plan geometry, all pointers device.
struct Geo {
    int NZ, NX, pitch, nb;
    int S;                         // shots of this launch (a batch); field buffers hold them at s * field
    int shot0;                     // global index of the batch's first shot (per-shot tables are global)
    int s_off;                     // batch-local index of this launch's first shot (a lane of the batch)
    int tz;                        // tile rows of the per-step kernels
    int nt_min;                    // shortest record of the batch: every shot is active below it
    int *err;                      // error word (bit 2: a bounded wait ran out)
    int ntz, ntx, ntiles;          // tiles per shot along z, x; total
    long long field;               // floats per shot field (NZ * pitch)
    // The Laplacian is evaluated as T = rz*S_z + S_x with integer weights
    // (5040 x the 8th-order weights), so that L u = T / (5040 dx^2) and
    // W (L u + s) = Wt T with Wt = dt^2 / (5040 dx^2 m) stored per cell as
    // the FP32 pair Wh + Wl (FP64-derived; Wl at Wh + field).
    float rz;                      // dx^2 / dz^2
    float iscale;                  // -1/dt^2: FWI imaging scale -1/m = iscale * 5040 dx^2 Wt
    float tscale;                  // 1 / (5040 dx^2): T -> L u + s
    float inj_scale;               // 5040 dx^2: residual r -> its T units
    const int *nt;                 // [S] record length
    const int *src_pt;             // [S] padded source point iz*pitch + ix
    const float *ws;               // [nt_max] 5040 dx^2 w(t_n) / (dx dz)
    const float *dGz, *dGx;        // [NZ], [pitch] 1 - g(d) of the sponge (1 beyond NX)
    const int *trec_off;           // [S*ntiles + 1] receivers per (shot, tile)
    const int *trec_pt;            // padded point of each receiver
    const int *trec_col;           // receiver index within its shot
    const long long *tr_off;       // [S] trace offsets
    const int *nrec;               // [S]
};

// One forward step n -> n+1 for all shots.  Field pointers are slot bases
// (shot s at + s*field).  u_next may alias u_prev (in-place update).
struct FwdArgs {
    const float *W;                // Wh [NZ][pitch], then Wl (padded, extension E applied)
    int cur_slot;                  // slot of u^n in the (halo) tile map
    int prev_slot;                 // slot of u^{n-1} in the interior map
    float *u_next;
    float *ck_cur, *ck_prev;       // checkpoint targets for (u^n, u^{n-1}) or null
    float *traces;                 // gather target (CSR) or null
    float *t_out;                  // T^n = 5040 dx^2 (L u^n + s^n) target (slot base) or null
    int n;
};

// Born step: background u and scattered du together (eq. Born).
// Two forward steps n, n+1 in one launch (full history): reads u^{n-1},
// u^n from fbuf slots, writes u^{n+1}, u^{n+2} to the other two (out of
// place: neighbouring CTAs read u^{n-1} and u^n around their own tiles).
struct Fwd2Args {
    const float *W;
    int prev_slot, cur_slot;       // u^{n-1} (4-cell halo map), u^n (8-cell halo map)
    float *u1, *u2;                // out: u^{n+1}, u^{n+2}
    float *traces;                 // CSR traces or null
    float *t1, *t2;                // out: T^n, T^{n+1} (history slots n+1, n+2)
    int n;
};

struct BornArgs {
    const float *W, *rho;
    int u_slot;                    // slot of u^n in the u tile map
    const float *u_prev;
    float *u_next;
    int d_slot;                    // slot of du^n in the du tile map
    const float *d_prev;
    float *d_next;
    int u_prev_slot, d_prev_slot;  // slots of u^{n-1}, du^{n-1} in the interior maps
    float *ck_cur, *ck_prev;
    float *traces;                 // scattered-field gather
    float *t_out;                  // T^n of the background field (slot base) or null
    int n;
};

// Adjoint step n (z^n from z^{n+1}, z^{n+2}) fused with the imaging condition
// img += scale * z^n * (L u^n + s^n), scale = -1/m (FWI) or -1 (Born), with
// L u^n + s^n read as the forward sweep's stored T^n / (5040 dx^2).
struct AdjArgs {
    const float *W;
    int z1_slot;                   // slot of z^{n+1} in the z (halo) tile map
    int z2_slot;                   // slot of z^{n+2} in the z interior map
    float *z2n;                    // out: z^n over z^{n+2} (same cells)
    int t_slot;                    // slot of T^n in the T interior map
    const float *resid;            // CSR residual traces
    float *img;                    // per-shot accumulators [S][field]
    int n;
    int born;
    int t_early;                   // T^n is not written by the preceding launches: copy it before the grid wait
};

// Number of kernels this library has launched (host-side count).
extern std::atomic<unsigned long long> g_launch_count;
// While a sweep is being captured into a CUDA graph its launches are counted
// here instead (the graph adds them to g_launch_count each time it runs).
extern thread_local unsigned long long *g_capture_count;
inline void count_launch(unsigned n = 1)
{
    if (g_capture_count) *g_capture_count += n;
    else g_launch_count.fetch_add(n, std::memory_order_relaxed);
}

// Message returned by aafwi_last_error(NULL) for calls made without a plan.
void set_call_error(const std::string &msg);

// Workspace layout of a plan (api.cu): shots per batch, full history or
// checkpoints, bytes against the budget (opts or 85 % of free memory).
struct PlanLayout {
    int Sb, nbatch;
    bool full;
    int k, nck;
    size_t bytes, budget;
    bool fits;
};
// U-Net kernels' error word (bit 0: a tensor-core wait ran out), read and cleared; -1 if unreadable.
int unet_take_error();

PlanLayout plan_layout(long long field, long long cells, int S, int nt_max, long long trace_count,
                       const aafwi_plan_opts &o);

cudaError_t init_kernels();  // per-device kernel attributes (dynamic shared memory)
void launch_prep(const Geo &g, int nz, int nx, const float *m, const float *rho, float mcfl,
                 double K, float *W, float *rho_pad, int *err, cudaStream_t st);
// Step launches with pdl = true may become resident while the previous
// kernel in the stream drains (programmatic dependent launch); they touch no
// memory written by earlier launches before their grid-dependency wait.
// tm_w: the model pair (Wh, Wl) as slots 0 and 1 of a one-shot interior map.
void launch_fwd(const Geo &g, const FwdArgs &a, const CUtensorMap &tm_u, const CUtensorMap &tm_p,
                const CUtensorMap &tm_w, cudaStream_t st, bool pdl = false);
void launch_fwd2(const Geo &g, const Fwd2Args &a, const CUtensorMap &tm_u8, const CUtensorMap &tm_u4, cudaStream_t st,
                 bool pdl = false);
void launch_born(const Geo &g, const BornArgs &a, const CUtensorMap &tm_u, const CUtensorMap &tm_d,
                 const CUtensorMap &tm_ui, const CUtensorMap &tm_di, const CUtensorMap &tm_w, const CUtensorMap &tm_r,
                 cudaStream_t st, bool pdl);
void launch_adj(const Geo &g, const AdjArgs &a, const CUtensorMap &tm_z, const CUtensorMap &tm_z2,
                const CUtensorMap &tm_t, const CUtensorMap &tm_w, cudaStream_t st, bool pdl = false);
// Shot sum and E^T of the batch's images: rowsum (FP64 [NZ][nx]) = or +=
// (accumulate) the sum over the batch's shots; the second pass, when out is
// not null, folds rowsum over z into out [nz][nx].
void launch_shot_sum(const Geo &g, int nz, int nx, const float *img, double *rowsum, bool accumulate, float *out,
                     cudaStream_t st);

// Persistent sweeps (persist_kernels.cu): one cooperative launch per sweep,
// one CTA per strip of rows, (pitch/4) x ty threads (at most PT): thread
// (x, y) owns float4 column x of the y-th block of the strip's rows.
constexpr int PT = 448;            // 14 warps: up to 144 registers a thread
constexpr int RBMAX = 12;          // rows per thread (the row loop is unrolled)
struct PGeo {
    int P;                         // strips (CTAs)
    int rows_max;                  // max rows of a strip
    int ty;                        // thread rows per CTA
    int slots_max;                 // max receiver slots of a strip
    long long slot;                // floats per history slot (S * field)
    const int *row0;               // [P+1] strip row ranges in global rows (shot * NZ + z)
    const int *grp_slot;           // [S*NZ*pitch/4] receiver slot of a float4 group, or -1
    const int *slot_off;           // [P+1] slots of each strip
    const int *slot_group;         // [slots] global group index of a slot
    const int4 *slot_cols;         // [slots] receiver index per lane (-1: none)
    float *exch;                   // [2][P][8][pitch] strip edge rows
    unsigned *flags;               // [P] completed steps of each strip
    int *err;                      // bit 2: a bounded wait ran out
};
struct PFwdArgs {
    const float *W;                // Wh, Wl as in FwdArgs
    float *hist;                   // slot n+1 <- T^n = 5040 dx^2 (L u^n + s^n); slot 0 untouched
    float *traces;                 // CSR gather target or null
    int nt;                        // steps (max over shots)
    int stall_step;                // test hook: strip 0 stops publishing at this step (-1: never)
};
struct PAdjArgs {
    const float *W;
    const float *hist;             // T^n (slot n+1) from the forward sweep
    const float *resid;            // CSR residual traces
    float *img;                    // per-shot accumulators [S][field]
    int nt;
    int born;
    int stall_step;                // test hook, as in PFwdArgs
};
size_t persist_smem(const Geo &g, int rows_max, int slots_max);
cudaError_t init_persist_kernels(size_t smem);
cudaError_t launch_fwd_persist(const Geo &g, const PGeo &pg, const PFwdArgs &a, size_t smem, cudaStream_t st);
cudaError_t launch_adj_persist(const Geo &g, const PGeo &pg, const PAdjArgs &a, size_t smem, cudaStream_t st);

// Reductions (FP64 accumulation, deterministic two-pass).
constexpr int RED_BLOCKS = 608;    // 4 x 152 SMs
void launch_misfit(const float *d_syn, const float *d_obs, float *resid, long long n,
                   double *partials, double *J_dev, cudaStream_t st);
void launch_absmax(const float *x, long long n, double *partials, double *out_dev, cudaStream_t st);
void launch_dot(const float *x, const float *y, long long n, double *partials, double *out_dev, cudaStream_t st);
void launch_axpby(float a, const float *x, float b, float *y, long long n, cudaStream_t st, float lo = 0.f,
                  float hi = 0.f);

// Anderson acceleration.
constexpr int AA_MAXM = 20;
constexpr int AA_LP_ROWS = 4096;        // rows one l-infinity round may add to its working set
constexpr int AA_LP_MAX_ROUNDS = 3000;  // rounds of the l1 / l-infinity LP before giving up
constexpr double AA_LP_GAP = 1e-9;      // relative optimality gap at which the LP rounds stop
struct AALpStats {
    double objective = 0.0, lower_bound = 0.0;
    int rounds = 0, rows = 0;
};
struct AAState {
    long long n;
    int M;
    float *ring_p, *ring_g;        // [M+1][n]
    double *gram;                  // [(M+1)*(M+1)]: H = dG^T dG by the slots naming the differences
    double *partials;              // [RED_BLOCKS][2 * AA_MAXM] (aa_step), [RED_BLOCKS] (combine)
    double *gamma;                 // [M]
    int *meta;                     // [0] Mk used, [1] first dropped column
    double *dot;                   // [1] armijo dot
    double eta;
    double beta;                   // damping of the AA point (1: Alg. 2)
    float *weights;                // [n] diagonal weights of a weighted l2 norm, or null
    int count, head;               // entries in the ring, slot of the newest
    int norm;                      // AAFWI_NORM_L2 / _L1 / _LINF
    int *lp_rows, *lp_cnt;         // l1 / l-infinity rounds: rows above a level [AA_LP_ROWS], their count
    double *lp_part, *lp_gat;      // per-block partials [RED_BLOCKS][AA_MAXM+1], gathered rows
    AALpStats lp;                  // of the last l1 / l-infinity step
    int slots[AA_MAXM + 1];        // chronological slots of the last step's window
};
// Alg. 2 steps 1-3: append (p_k, G_k) and solve the l2 least squares for gamma
// (the rank safeguard decides the kept columns)...
void launch_aa_step(AAState &s, const float *p_k, const float *g_k, cudaStream_t st);
// ...then form p_tilde, p_bar from the gamma in s.gamma.
void launch_aa_mix(AAState &s, float *p_tilde, float *p_bar, cudaStream_t st);
void launch_aa_combine(AAState &s, float lam, const float *p_tilde, const float *p_bar,
                       float *p_next, float lo, float hi, bool want_dot, cudaStream_t st);
// l1 / l-infinity gamma over the kept window slots[0..mk] (host rounds over
// device passes; gamma_in: the l2 solution); AAFWI_OK or an error (msg set).
int aa_lp_gamma(AAState &s, const int *slots, int mk, int norm, const double *gamma_in, double *gamma,
                AALpStats *stats, std::string *msg, cudaStream_t st);

}  // namespace aafwi
