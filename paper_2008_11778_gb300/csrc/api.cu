// api.cu -- the C ABI of include/aafwi.h: plans (geometry, workspace,
// wavefield history or checkpoints), the forward / Born / adjoint sweeps that
// drive the time-step kernels, the misfit, and the Anderson-acceleration
// state.  Host code only orchestrates; every arithmetic step runs in the
// kernels of wave_kernels.cu and reduce_kernels.cu.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>
#include <set>
#include <mutex>

#include "../../include/aafwi.h"
#include "internal.cuh"

using namespace aafwi;

namespace {

thread_local std::string g_create_error;
constexpr double kCflLimit = 0.55;
constexpr double kSpongeA = 0.015;

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

constexpr int kMaxLanes = 8;   // shot lanes of a per-step sweep: the caller's stream + 7 lane streams

struct aafwi_plan {
    int device = 0;
    int nx = 0, nz = 0, nb = 0, NZ = 0, NX = 0, pitch = 0, S = 0, nt_max = 0;
    int Sb = 0, nbatch = 1;         // shots per batch (the wavefield buffers hold Sb shots), batches
    double dx = 0, dz = 0, dt = 0;
    std::vector<int> nt;
    std::vector<long long> tr_off;
    long long trace_count = 0;
    long long field = 0;            // floats per shot field
    int k = 1, nck = 0;             // checkpoint interval (1: full history), count
    bool full = true;
    Geo geo{};
    std::vector<Buf> bufs;
    // device buffers
    float *W = nullptr, *rho_pad = nullptr;   // W: Wh then Wl, each [NZ][pitch]
    double K = 0.0;                 // dt^2 / (5040 dx^2)
    float *hist = nullptr;          // full: T^n in slot n+1 (nt_max+1 slots); else 2*nck checkpoint slots
    float *fbuf = nullptr;          // 4 forward slots: one-step sweeps rotate u^n, u^{n-1} in slots 0, 1
                                    // (in place); two-step sweeps alternate pairs (0, 1) and (2, 3)
    float *rbuf = nullptr;          // k replay slots of T (checkpoint mode)
    float *dbuf = nullptr;          // 2 rotating Born slots
    float *zbuf = nullptr;          // 2 rotating adjoint slots
    float *img = nullptr;           // per-shot image accumulators
    // TMA descriptors of the buffers the per-step kernels stage from: halo
    // boxes of fbuf, dbuf, zbuf and the checkpoints; interior boxes of fbuf,
    // zbuf, the checkpoints and the T history / replay buffer
    CUtensorMap tm_f{}, tm_d{}, tm_z{}, tm_ck{};
    CUtensorMap tm_fi{}, tm_zi{}, tm_cki{}, tm_t{};
    CUtensorMap tm_w{};             // (Wh, Wl) as slots 0, 1 of a one-shot map
    CUtensorMap tm_di{}, tm_rho{};  // interior boxes of dbuf; rho_pad as a one-shot, one-slot map
    CUtensorMap tm_f8{};            // fbuf with an 8-cell halo (two-step forward)
    float *dsyn = nullptr, *resid = nullptr;
    // device staging of aafwi_adjoint_gradient_host (allocated on first use)
    float *stage_m = nullptr, *stage_rho = nullptr, *stage_d = nullptr, *stage_g = nullptr;
    double *partials = nullptr, *J = nullptr;
    double *rowsum = nullptr;       // [NZ][nx] FP64 partial sums of the shot sum
    int *err = nullptr;
    size_t ws_bytes = 0;
    bool fwd_valid = false;
    const float *fwd_model = nullptr;
    bool retired = false;           // a TMA wait ran out: every later call is refused
    // persistent engine
    bool persist_fwd = false;       // FWI forward sweeps: one cooperative launch each
    bool persist_adj = false;       // adjoint sweeps: one cooperative launch each
    bool hist_T = false;            // the history holds T^n of the last forward sweep
    PGeo pgeo{};
    size_t psmem = 0;
    int stall_step = -1;            // test hook (aafwi_plan_set_stall)
    // CUDA graphs of the per-step sweeps (one launch per time step): each
    // (sweep kind, caller buffer) is captured once and then replayed
    bool graphs = true;
    bool pdl = true;   // per-step launches after a sweep's first: programmatic dependents
    int steps_per_launch = 1;       // full-history FWI forward sweeps: 1 or 2 (k_fwd2)
    struct SweepGraph {
        int kind;                   // SWEEP_*
        const void *ptr;            // the caller buffer the sweep reads or writes
        cudaGraphExec_t exec;
        unsigned long long kernels; // kernel launches per replay
    };
    std::vector<SweepGraph> sweep_graphs;   // most recently used last
    cudaStream_t cap = nullptr;     // capture stream
    // shot lanes: the per-step sweeps of a batch run as `lanes` independent
    // launch chains over consecutive shot groups, on forked streams
    int lanes = 4;
    cudaStream_t lane_st[kMaxLanes - 1] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kMaxLanes - 1] = {};
    ~aafwi_plan()
    {
        for (cudaStream_t s : lane_st)
            if (s) cudaStreamDestroy(s);
        for (cudaEvent_t e : ev_join)
            if (e) cudaEventDestroy(e);
        if (ev_fork) cudaEventDestroy(ev_fork);
    }
    std::string msg;
};

struct aafwi_aa {
    AAState s{};
    float *wbuf = nullptr;          // copy of the weighted-l2 weights
    int device = 0;
    std::vector<Buf> bufs;
};

namespace {

int fail(aafwi_plan *p, int code, const std::string &m)
{
    if (p) p->msg = m;
    else g_create_error = m;
    return code;
}

int cuda_fail(aafwi_plan *p, cudaError_t e, const char *what)
{
    return fail(p, AAFWI_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <class T>
bool dalloc(std::vector<Buf> &bufs, T **out, size_t count)
{
    void *p = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    bufs.push_back({p, bytes});
    if (cudaMemset(p, 0, bytes) != cudaSuccess) return false;   // u^0 = 0, zero pitch padding
    *out = static_cast<T *>(p);
    return true;
}

void free_bufs(std::vector<Buf> &bufs)
{
    for (auto &b : bufs) cudaFree(b.p);
    bufs.clear();
}

template <class T>
bool upload(std::vector<Buf> &bufs, T **out, const std::vector<T> &h)
{
    if (!dalloc(bufs, out, h.size())) return false;
    return cudaMemcpy(*out, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
}

float *slot(float *base, long long per_slot, long long i) { return base + per_slot * i; }

// Sweep kinds of the graph cache; SWEEP_FWD_TRACES is a forward sweep that
// stores no history (the traces of a plan whose history cannot be reused).
enum { SWEEP_FWD = 0, SWEEP_BORN = 1, SWEEP_ADJ = 2, SWEEP_ADJ_BORN = 3, SWEEP_FWD_TRACES = 4, SWEEP_KINDS = 5 };
constexpr size_t kMaxSweepGraphs = 8;   // per batch

void drop_graphs(aafwi_plan *p)
{
    for (auto &gr : p->sweep_graphs) cudaGraphExecDestroy(gr.exec);
    p->sweep_graphs.clear();
    if (p->cap) cudaStreamDestroy(p->cap);
    p->cap = nullptr;
}

constexpr int kDefaultLanes = 4;

// Scratch of the stand-alone reductions (aafwi_dot, aafwi_absmax): RED_BLOCKS
// FP64 partials and the result, allocated once per device on first use and
// reused by every later call.  Callers hold g_red_mu until the result is back
// on the host, so calls from several host threads do not share it in flight.
std::mutex g_red_mu;
constexpr int kMaxDevices = 64;
double *g_red_buf[kMaxDevices] = {};

bool reduction_scratch(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return false;
    if (!g_red_buf[dev] && cudaMalloc((void **)&g_red_buf[dev], (RED_BLOCKS + 1) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        g_red_buf[dev] = nullptr;
        return false;
    }
    *out = g_red_buf[dev];
    return true;
}

// The batch's shots split into p->lanes consecutive groups (fewer if the
// batch has fewer shots), each with its launch geometry and stream: lane 0
// on st, the others on the plan's lane streams forked from st.  One lane's
// step boundary (grid drain, dependency, refill) then overlaps the other
// lanes' work.  Lanes touch disjoint shots, so results do not depend on
// how their launches interleave.
struct Lanes {
    int L = 1;
    Geo g[kMaxLanes];
    cudaStream_t st[kMaxLanes];
};

int fork_lanes(aafwi_plan *p, const Geo &g, cudaStream_t st, Lanes &ln)
{
    ln.L = std::max(1, std::min(p->lanes, g.S));
    int off = 0;
    for (int l = 0; l < ln.L; ++l) {
        const int cnt = g.S / ln.L + (l < g.S % ln.L ? 1 : 0);
        ln.g[l] = g;
        ln.g[l].s_off = g.s_off + off;
        ln.g[l].S = cnt;
        ln.st[l] = l == 0 ? st : p->lane_st[l - 1];
        off += cnt;
    }
    if (ln.L == 1) return AAFWI_OK;
    cudaError_t e = cudaEventRecord(p->ev_fork, st);
    for (int l = 1; l < ln.L && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(ln.st[l], p->ev_fork, 0);
    return e == cudaSuccess ? AAFWI_OK : cuda_fail(p, e, "lane fork");
}

int join_lanes(aafwi_plan *p, const Lanes &ln)
{
    cudaError_t e = cudaSuccess;
    for (int l = 1; l < ln.L && e == cudaSuccess; ++l) {
        e = cudaEventRecord(p->ev_join[l - 1], ln.st[l]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ln.st[0], p->ev_join[l - 1], 0);
    }
    return e == cudaSuccess ? AAFWI_OK : cuda_fail(p, e, "lane join");
}

// Run body(stream) -- a sweep of per-step launches -- through the plan's
// graph cache: capture it on the plan's capture stream the first time this
// (kind, ptr) is seen, then replay the instantiated graph on st.
template <class F>
int run_graph(aafwi_plan *p, int kind, const void *ptr, cudaStream_t st, F body)
{
    auto &gs = p->sweep_graphs;
    size_t i = 0;
    while (i < gs.size() && !(gs[i].kind == kind && gs[i].ptr == ptr)) ++i;
    if (i == gs.size()) {
        if (!p->cap && cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess)
            return cuda_fail(p, cudaGetLastError(), "capture stream");
        unsigned long long kernels = 0;
        cudaError_t e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(p, e, "begin capture");
        g_capture_count = &kernels;
        const int rc = body(p->cap);
        g_capture_count = nullptr;
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(p->cap, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(p, e, "end capture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(p, e, "graph instantiate");
        if (gs.size() >= kMaxSweepGraphs * (size_t)p->nbatch) {
            cudaGraphExecDestroy(gs.front().exec);
            gs.erase(gs.begin());
        }
        gs.push_back({kind, ptr, exec, kernels});
        i = gs.size() - 1;
    } else if (i + 1 != gs.size()) {
        std::rotate(gs.begin() + i, gs.begin() + i + 1, gs.end());   // most recently used last
        i = gs.size() - 1;
    }
    cudaError_t e = cudaGraphLaunch(gs[i].exec, st);
    if (e != cudaSuccess) return cuda_fail(p, e, "graph launch");
    count_launch((unsigned)gs[i].kernels);
    return AAFWI_OK;
}

int check_launch(aafwi_plan *p)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(p, e, "kernel launch");
    return AAFWI_OK;
}

int run_persist_forward(aafwi_plan *p, float *traces, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(p->pgeo.flags, 0, p->pgeo.P * sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_fail(p, e, "memset");
    PFwdArgs a{p->W, p->hist, traces, p->nt_max, p->stall_step};
    e = launch_fwd_persist(p->geo, p->pgeo, a, p->psmem, st);
    if (e != cudaSuccess) return cuda_fail(p, e, "persistent forward launch");
    return AAFWI_OK;
}

// Geometry of batch b (shots b*Sb .. ; the per-shot tables stay global).
Geo batch_geo(const aafwi_plan *p, int b)
{
    Geo g = p->geo;
    g.shot0 = b * p->Sb;
    g.S = std::min(p->Sb, p->S - g.shot0);
    g.nt_min = *std::min_element(p->nt.begin() + g.shot0, p->nt.begin() + g.shot0 + g.S);
    return g;
}

// Per-step forward sweep over the batch's shots (born: u and du together).
// u^n and u^{n-1} rotate in fbuf (u^{n+1} overwrites u^{n-1} in place); with
// the full history T^n goes to history slot n+1, else (u^n, u^{n-1}) are
// checkpointed every k steps.  With store = false neither is written (the
// traces alone are wanted).
int sweep_forward(aafwi_plan *p, const Geo &g, bool born, bool store, float *traces, cudaStream_t st)
{
    const long long ps = (long long)p->Sb * p->field;
    if (cudaMemsetAsync(p->fbuf, 0, 2 * ps * sizeof(float), st) != cudaSuccess)
        return cuda_fail(p, cudaGetLastError(), "memset");
    if (born && cudaMemsetAsync(p->dbuf, 0, 2 * ps * sizeof(float), st) != cudaSuccess)
        return cuda_fail(p, cudaGetLastError(), "memset");
    Lanes ln;
    int rc = fork_lanes(p, g, st, ln);
    if (rc) return rc;
    int n0 = 0, cur = 0, prv = 1;   // after the two-step part: u^n in slot cur, u^{n-1} in slot prv
    if (!born && p->full && p->steps_per_launch == 2) {
        // (u^{n-1}, u^n) in slots (2q, 2q+1); (u^{n+1}, u^{n+2}) to the other pair
        int q = 0;
        for (; n0 + 1 < p->nt_max; n0 += 2, q ^= 1) {
            Fwd2Args a{p->W, 2 * q, 2 * q + 1, slot(p->fbuf, ps, 2 * (q ^ 1)), slot(p->fbuf, ps, 2 * (q ^ 1) + 1),
                       traces, store ? slot(p->hist, ps, n0 + 1) : nullptr,
                       store ? slot(p->hist, ps, n0 + 2) : nullptr, n0};
            for (int l = 0; l < ln.L; ++l) launch_fwd2(ln.g[l], a, p->tm_f8, p->tm_f, ln.st[l], p->pdl && n0 > 0);
        }
        cur = 2 * q + 1;
        prv = 2 * q;
    }
    for (int n = n0; n < p->nt_max; ++n) {
        // one step: u^{n+1} overwrites u^{n-1} in place, then the slots swap roles
        float *prev = slot(p->fbuf, ps, prv), *next = prev;
        float *ckc = nullptr, *ckp = nullptr, *tout = nullptr;
        if (!store) {
        } else if (p->full) {
            tout = slot(p->hist, ps, n + 1);
        } else if (n % p->k == 0) {
            ckc = slot(p->hist, ps, 2LL * (n / p->k));
            ckp = slot(p->hist, ps, 2LL * (n / p->k) + 1);
        }
        for (int l = 0; l < ln.L; ++l) {
            if (born) {
                BornArgs a{p->W, p->rho_pad, cur, prev, next, n & 1,
                           slot(p->dbuf, ps, (n + 1) & 1), slot(p->dbuf, ps, (n + 1) & 1), prv, (n + 1) & 1,
                           ckc, ckp, traces, tout, n};
                launch_born(ln.g[l], a, p->tm_f, p->tm_d, p->tm_fi, p->tm_di, p->tm_w, p->tm_rho, ln.st[l],
                            p->pdl && n > 0);
            } else {
                FwdArgs a{p->W, cur, prv, next, ckc, ckp, traces, tout, n};
                launch_fwd(ln.g[l], a, p->tm_f, p->tm_fi, p->tm_w, ln.st[l], p->pdl && n > 0);
            }
        }
        std::swap(cur, prv);
    }
    rc = join_lanes(p, ln);
    if (rc) return rc;
    return check_launch(p);
}

// Forward sweep over batch b (born: u and du together); traces -> CSR.
// store = false: no history or checkpoints (FWI forward of per-step engines).
int run_forward(aafwi_plan *p, int b, bool born, float *traces, cudaStream_t st, bool store = true)
{
    p->hist_T = false;
    int rc;
    const Geo g = batch_geo(p, b);
    store = store || born || p->persist_fwd;
    if (p->persist_fwd && !born) rc = run_persist_forward(p, traces, st);
    else if (!p->graphs) rc = sweep_forward(p, g, born, store, traces, st);
    else
        rc = run_graph(p, (born ? SWEEP_BORN : store ? SWEEP_FWD : SWEEP_FWD_TRACES) + SWEEP_KINDS * b, traces, st,
                       [&](cudaStream_t cs) { return sweep_forward(p, g, born, store, traces, cs); });
    p->hist_T = rc == AAFWI_OK && p->full && store;
    return rc;
}

// Per-step adjoint sweep with imaging into p->img (checkpoint mode: segment
// replays from the stored checkpoints in between).
int sweep_adjoint(aafwi_plan *p, const Geo &g, bool born, const float *resid, cudaStream_t st)
{
    const long long ps = (long long)p->Sb * p->field;
    if (cudaMemsetAsync(p->img, 0, ps * sizeof(float), st) != cudaSuccess)
        return cuda_fail(p, cudaGetLastError(), "memset");
    if (cudaMemsetAsync(p->zbuf, 0, 2 * ps * sizeof(float), st) != cudaSuccess)
        return cuda_fail(p, cudaGetLastError(), "memset");
    // The first launch of each lane follows the memsets and runs as a plain
    // launch; every later step kernel follows a step kernel and is launched
    // as a programmatic dependent of it.  With the full history no launch of
    // the sweep writes T, so the adjoint copies T^n before its grid wait.
    Lanes ln;
    int rc = fork_lanes(p, g, st, ln);
    if (rc) return rc;
    bool first = true;
    auto adj = [&](int n, int t_slot) {   // T^n in slot t_slot of the T map
        AdjArgs a{p->W, (n + 1) & 1, n & 1, slot(p->zbuf, ps, n & 1), t_slot, resid, p->img, n, born ? 1 : 0,
                  p->full && !first ? 1 : 0};
        for (int l = 0; l < ln.L; ++l)
            launch_adj(ln.g[l], a, p->tm_z, p->tm_zi, p->tm_t, p->tm_w, ln.st[l], p->pdl && !first);
        first = false;
    };
    if (p->full) {
        for (int n = p->nt_max - 1; n >= 0; --n) adj(n, n + 1);
    } else {
        // segment j = steps [a, e): replay the forward from its checkpoint
        // (u^a, u^{a-1}) storing T^a .. T^{e-1} in rbuf, then step back
        // through it.  u^m, m > a, rotates in fbuf (checkpoints stay intact).
        for (int j = p->nck - 1; j >= 0; --j) {
            const int a = j * p->k, e = std::min(a + p->k, p->nt_max);
            // u^m: checkpoint slot 2j (m = a), 2j+1 (m = a-1), else fbuf slot m&1
            auto ck = [&](int m) { return m == a || m == a - 1; };
            auto uslot = [&](int m) { return m == a ? 2 * j : m == a - 1 ? 2 * j + 1 : (m & 1); };
            for (int n = a; n < e; ++n) {
                FwdArgs f{p->W, uslot(n), uslot(n - 1), slot(p->fbuf, ps, (n + 1) & 1), nullptr,
                          nullptr, nullptr, slot(p->rbuf, ps, n - a), n};
                for (int l = 0; l < ln.L; ++l)
                    launch_fwd(ln.g[l], f, ck(n) ? p->tm_ck : p->tm_f, ck(n - 1) ? p->tm_cki : p->tm_fi, p->tm_w,
                               ln.st[l], p->pdl && !first);
                first = false;
            }
            for (int n = e - 1; n >= a; --n) adj(n, n - a);
        }
    }
    rc = join_lanes(p, ln);
    if (rc) return rc;
    return check_launch(p);
}

// Adjoint sweep of batch b with imaging into p->img (born: scale -1, else -1/m).
int run_adjoint(aafwi_plan *p, int b, bool born, const float *resid, cudaStream_t st)
{
    if (p->persist_adj && p->hist_T) {
        const long long ps = (long long)p->Sb * p->field;
        if (cudaMemsetAsync(p->img, 0, ps * sizeof(float), st) != cudaSuccess)
            return cuda_fail(p, cudaGetLastError(), "memset");
        cudaError_t e = cudaMemsetAsync(p->pgeo.flags, 0, p->pgeo.P * sizeof(unsigned), st);
        if (e != cudaSuccess) return cuda_fail(p, e, "memset");
        PAdjArgs a{p->W, p->hist, resid, p->img, p->nt_max, born ? 1 : 0, p->stall_step};
        e = launch_adj_persist(p->geo, p->pgeo, a, p->psmem, st);
        if (e != cudaSuccess) return cuda_fail(p, e, "persistent adjoint launch");
        return AAFWI_OK;
    }
    const Geo g = batch_geo(p, b);
    if (!p->graphs) return sweep_adjoint(p, g, born, resid, st);
    return run_graph(p, (born ? SWEEP_ADJ_BORN : SWEEP_ADJ) + SWEEP_KINDS * b, resid, st,
                     [&](cudaStream_t cs) { return sweep_adjoint(p, g, born, resid, cs); });
}

int prep(aafwi_plan *p, const float *m, const float *rho, cudaStream_t st)
{
    const double h = std::min(p->dx, p->dz);
    const double mcfl = std::pow(p->dt / (kCflLimit * h), 2.0);  // m below this violates CFL
    launch_prep(p->geo, p->nz, p->nx, m, rho, (float)mcfl, p->K, p->W, rho ? p->rho_pad : nullptr,
                p->err, st);
    return check_launch(p);
}

constexpr const char *kRetired =
    "a tile copy (TMA) did not complete within its bounded wait; the plan is retired and refuses every "
    "later call: destroy it and reset the device context (cudaDeviceReset) before continuing";

// The first check of every plan entry point: a retired plan runs nothing.
int refuse_retired(aafwi_plan *p)
{
    return p && p->retired ? fail(p, AAFWI_ERR_TIMEOUT, kRetired) : AAFWI_OK;
}

int finish_sync(aafwi_plan *p, double *J_host, cudaStream_t st)
{
    if (!J_host) return AAFWI_OK;
    int err = 0;
    cudaError_t e = cudaMemcpyAsync(J_host, p->J, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, p->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(p, e, "synchronise");
    if (err) {
        p->fwd_valid = false;
        if (err & 8) {
            p->retired = true;
            return fail(p, AAFWI_ERR_TIMEOUT, kRetired);
        }
        cudaMemsetAsync(p->err, 0, sizeof(int), st);
        if (err & 1) return fail(p, AAFWI_ERR_NAN, "model has a non-finite or non-positive value");
        if (err & 4) return fail(p, AAFWI_ERR_TIMEOUT, "a persistent sweep's bounded wait ran out");
        return fail(p, AAFWI_ERR_CFL, "model velocity exceeds the CFL limit of the plan");
    }
    return AAFWI_OK;
}

// Decide which sweeps run persistently and build the strip tables.  Returns
// 0 (engine chosen) or an error code when PERSISTENT or HYBRID was required.
int setup_persist(aafwi_plan *p, int engine, const aafwi_shots *sh, std::string *why)
{
    p->persist_fwd = p->persist_adj = false;
    // AUTO takes the per-step engine: on every workload measured here it is the
    // fastest (aafwi_autotune decides per geometry when asked)
    if (engine == AAFWI_ENGINE_PER_STEP || engine == AAFWI_ENGINE_AUTO) return AAFWI_OK;
    auto no = [&](const char *m) {
        if (engine == AAFWI_ENGINE_PERSISTENT || engine == AAFWI_ENGINE_HYBRID) {
            *why = std::string("persistent engine not available: ") + m;
            return AAFWI_ERR_ARG;
        }
        return AAFWI_OK;
    };
    if (!p->full) return no("needs the full wavefield history");
    if (p->nbatch > 1) return no("the shots do not fit in one batch");
    int dev = 0, sms = 0, coop = 0, smem_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!coop || sms < 1) return no("cooperative launch unsupported");
    const int W4 = p->pitch / 4;
    if (W4 > PT) return no("rows wider than a CTA");
    const long long R = (long long)p->S * p->NZ;
    int P = (int)std::min<long long>(sms, R / 4);        // strips of at least 4 rows
    if (P < 1) return no("grid too small");
    const int rows_max = (int)((R + P - 1) / P);
    const int inner = std::max(0, rows_max - 8);           // rows of phase 1 (no halo)
    const int ty = std::max(1, std::min(PT / W4, std::max(1, inner)));
    if ((inner + ty - 1) / ty > RBMAX) return no("too many rows per thread");
    // strips and receiver slots
    std::vector<int> row0(P + 1);
    for (int c = 0; c <= P; ++c) row0[c] = (int)(R * c / P);
    std::vector<int> grp_slot((size_t)R * W4, -1);
    std::vector<std::vector<std::pair<long long, int4>>> per(P);   // (group, cols) per strip
    std::vector<std::vector<int>> idx(P);
    for (int s = 0; s < p->S; ++s) {
        for (int j = sh->rec_off[s]; j < sh->rec_off[s + 1]; ++j) {
            const long long gr = (long long)s * p->NZ + sh->rec_iz[j] + p->nb;
            const int px = sh->rec_ix[j] + p->nb;
            const long long grp = gr * W4 + px / 4;
            const int c = (int)(std::upper_bound(row0.begin(), row0.end(), (int)gr) - row0.begin()) - 1;
            int k = -1;
            for (size_t q = 0; q < per[c].size(); ++q)
                if (per[c][q].first == grp) k = (int)q;
            if (k < 0) {
                per[c].push_back({grp, make_int4(-1, -1, -1, -1)});
                k = (int)per[c].size() - 1;
            }
            int *lanes = &per[c][k].second.x;
            lanes[px % 4] = j - sh->rec_off[s];
        }
    }
    std::vector<int> slot_off(P + 1, 0), slot_group;
    std::vector<int4> slot_cols;
    int slots_max = 0;
    for (int c = 0; c < P; ++c) {
        for (auto &e : per[c]) {
            grp_slot[e.first] = (int)slot_group.size();
            slot_group.push_back((int)e.first);
            slot_cols.push_back(e.second);
        }
        slot_off[c + 1] = (int)slot_group.size();
        slots_max = std::max<int>(slots_max, (int)per[c].size());
    }
    const size_t smem = persist_smem(p->geo, rows_max, slots_max);
    if ((long long)smem > smem_optin) return no("strips do not fit shared memory");
    if (init_persist_kernels(smem) != cudaSuccess) {
        cudaGetLastError();
        return no("kernel attributes");
    }
    if (slot_group.empty()) {
        slot_group.push_back(0);
        slot_cols.push_back(make_int4(-1, -1, -1, -1));
    }
    PGeo &pg = p->pgeo;
    int *d_row0, *d_gs, *d_so, *d_sg;
    int4 *d_sc;
    bool ok = upload(p->bufs, &d_row0, row0) && upload(p->bufs, &d_gs, grp_slot) &&
              upload(p->bufs, &d_so, slot_off) && upload(p->bufs, &d_sg, slot_group) &&
              upload(p->bufs, &d_sc, slot_cols) &&
              dalloc(p->bufs, &pg.exch, (size_t)2 * P * 8 * p->pitch) && dalloc(p->bufs, &pg.flags, P);
    if (!ok) return no("allocation");
    pg.P = P;
    pg.rows_max = rows_max;
    pg.ty = ty;
    pg.slots_max = slots_max;
    pg.slot = (long long)p->S * p->field;
    pg.row0 = d_row0; pg.grp_slot = d_gs; pg.slot_off = d_so; pg.slot_group = d_sg; pg.slot_cols = d_sc;
    pg.err = p->err;
    p->psmem = smem;
    p->persist_fwd = engine != AAFWI_ENGINE_HYBRID;
    p->persist_adj = true;
    return AAFWI_OK;
}

}  // namespace

void aafwi::set_call_error(const std::string &msg) { g_create_error = msg; }

// Layout of a plan's workspace: how many shots the wavefield buffers hold
// (shot batches), full T history or checkpoints, and the bytes.
//   * Full history for all shots if it fits the budget.
//   * Else full history for batches of shots, if a batch still covers at
//     least kMinBatchCells grid points per time step (enough to fill the GPU):
//     no replay sweep is needed.
//   * Else checkpoints every k ~ sqrt(2 nt) steps for the largest batch that fits.
// opts.checkpoint_every = 1 forces the full history, >= 2 checkpoints every
// that many steps; opts.shots_per_batch > 0 fixes the batch size.
PlanLayout aafwi::plan_layout(long long field, long long cells, int S, int nt_max, long long trace_count,
                              const aafwi_plan_opts &o)
{
    constexpr long long kMinBatchCells = 4LL << 20;
    PlanLayout L{};
    // shots whose adjoint working set (3 fields each) fits 40 % of the L2
    int l2_shots = 1;
    {
        int dev = 0, l2 = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess &&
            l2 > 0)
            l2_shots = std::max(1, (int)(0.4 * (double)l2 / (3.0 * (double)field * sizeof(float))));
        else
            cudaGetLastError();
    }
    size_t budget = o.max_workspace_bytes;
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        budget = (size_t)(0.85 * (double)fr);
    }
    L.budget = budget;
    const size_t F = (size_t)field * sizeof(float);
    auto fixed = [&](int Sb) {   // W pair + rho; fbuf (4 slots), dbuf, zbuf (2 each) + img; dsyn + resid
        return 3 * F + (4 + 2 + 2 + 1) * F * Sb + 2 * (size_t)trace_count * sizeof(float) + (1 << 20);
    };
    const int k = o.checkpoint_every >= 2 ? o.checkpoint_every
                                          : std::max(2, (int)std::lround(std::sqrt(2.0 * nt_max)));
    const int nck = (nt_max + k - 1) / k;
    auto full_bytes = [&](int Sb) { return fixed(Sb) + (size_t)(nt_max + 1) * F * Sb; };
    auto ck_bytes = [&](int Sb) { return fixed(Sb) + (size_t)(2 * nck + k) * F * Sb; };
    auto take = [&](int Sb, bool full) {
        L.Sb = Sb;
        L.nbatch = (S + Sb - 1) / Sb;
        L.full = full;
        L.k = full ? 1 : k;
        L.nck = full ? 0 : nck;
        L.bytes = full ? full_bytes(Sb) : ck_bytes(Sb);
        L.fits = L.bytes <= budget;
        return L;
    };
    std::vector<int> sizes;   // candidate batch sizes, largest first
    if (o.shots_per_batch > 0) {
        sizes.push_back(std::min(S, o.shots_per_batch));
    } else {
        for (int nb = 1; nb <= S; ++nb) {
            const int Sb = (S + nb - 1) / nb;
            if (sizes.empty() || Sb != sizes.back()) sizes.push_back(Sb);
        }
    }
    // A plan that runs its shots in batches anyway gains nothing from large
    // batches, but its per-step working set must stay in L2: the adjoint step
    // keeps z^{n+1}, z^{n+2} and the image of every shot of the batch in
    // flight, so batches hold at most l2_shots shots (measured on the large
    // workload, 2001 x 601: 3 shots per batch instead of 7 cut the
    // gradient's time per update by a quarter).  With opts.l2_batches = 1
    // a plan that would fit in one batch is split too (LSRTM gradients, which
    // reuse no stored forward: 4 batches of 16 shots instead of one of 64
    // cut the 737 x 240 gradient from 472 to 393 ms).
    auto l2_cap = [&](PlanLayout l) {
        if (o.shots_per_batch > 0 || o.l2_batches < 0 || (o.l2_batches == 0 && l.nbatch == 1) ||
            l.Sb <= l2_shots)
            return l;
        const int nb = (S + l2_shots - 1) / l2_shots;   // even split into the fewest batches that fit
        return take((S + nb - 1) / nb, l.full);
    };
    if (o.checkpoint_every <= 1) {
        for (int Sb : sizes)
            if (full_bytes(Sb) <= budget &&
                (o.checkpoint_every == 1 || Sb == S || Sb == sizes.front() || Sb * cells >= kMinBatchCells))
                return l2_cap(take(Sb, true));
        if (o.checkpoint_every == 1) return take(sizes.back(), true);   // does not fit: reported by the caller
    }
    for (int Sb : sizes)
        if (ck_bytes(Sb) <= budget) return l2_cap(take(Sb, false));
    return take(sizes.back(), false);
}

extern "C" {

const char *aafwi_last_error(const aafwi_plan *plan)
{
    return plan ? plan->msg.c_str() : g_create_error.c_str();
}

int aafwi_plan_create(const aafwi_grid *g, const aafwi_shots *sh, const double *wavelet,
                      const aafwi_plan_opts *opts, aafwi_plan **out)
{
    if (!g || !sh || !wavelet || !out) return fail(nullptr, AAFWI_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (g->nx < 1 || g->nz < 1 || g->nb < 0 || !(g->dx > 0) || !(g->dz > 0) || !(g->dt > 0) ||
        sh->S < 1 || !sh->src_iz || !sh->src_ix || !sh->nt || !sh->rec_off || !sh->rec_iz || !sh->rec_ix)
        return fail(nullptr, AAFWI_ERR_ARG, "invalid grid or shot description");
    const double h = std::min(g->dx, g->dz);
    if (!(g->c_max > 0) || g->c_max * g->dt / h > kCflLimit) {
        char b[160];
        snprintf(b, sizeof b, "CFL number c_max*dt/h = %.4f exceeds %.2f", g->c_max * g->dt / h, kCflLimit);
        return fail(nullptr, AAFWI_ERR_CFL, b);
    }
    aafwi_plan_opts o{};
    if (opts) o = *opts;
    // options and shapes are checked before any device call
    if (o.steps_per_launch < 0 || o.steps_per_launch > 2)
        return fail(nullptr, AAFWI_ERR_ARG, "steps_per_launch must be 0, 1 or 2");
    if (o.lanes < 0 || o.lanes > kMaxLanes) return fail(nullptr, AAFWI_ERR_ARG, "lanes must be 0 .. 8");
    if (o.tile_z != 0 && !tile_z_supported(o.tile_z))
        return fail(nullptr, AAFWI_ERR_ARG, "tile_z must be 0 (default), 16, 32 or 64");
    if (o.tile_x != 0 && o.tile_x != TX) return fail(nullptr, AAFWI_ERR_ARG, "tile_x must be 0 (default) or 128");
    if ((long long)(g->nz + 2 * g->nb) * ((g->nx + 2 * g->nb + 31) / 32 * 32) >= (1LL << 31))
        return fail(nullptr, AAFWI_ERR_ARG, "padded grid of 2^31 cells or more");   // 32-bit cell offsets
    if (*std::min_element(sh->nt, sh->nt + sh->S) < 1) return fail(nullptr, AAFWI_ERR_ARG, "record length must be >= 1");
    if (sh->rec_off[0] != 0) return fail(nullptr, AAFWI_ERR_ARG, "rec_off[0] must be 0");
    {
        cudaError_t ie = init_kernels();
        if (ie != cudaSuccess) return cuda_fail(nullptr, ie, "kernel attributes");
    }
    auto *p = new aafwi_plan();
    cudaGetDevice(&p->device);
    p->graphs = o.no_graphs == 0;
    p->pdl = o.no_pdl == 0;
    p->steps_per_launch = o.steps_per_launch == 2 ? 2 : 1;
    p->lanes = o.lanes == 0 ? kDefaultLanes : o.lanes;
    if (p->lanes > 1) {
        bool ok = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) == cudaSuccess;
        for (int l = 0; ok && l + 1 < p->lanes; ++l)
            ok = cudaStreamCreateWithFlags(&p->lane_st[l], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&p->ev_join[l], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            delete p;   // the destructor releases the streams and events made so far
            return cuda_fail(nullptr, cudaGetLastError(), "lane streams");
        }
    }
    p->nx = g->nx; p->nz = g->nz; p->nb = g->nb;
    p->dx = g->dx; p->dz = g->dz; p->dt = g->dt;
    p->NZ = g->nz + 2 * g->nb;
    p->NX = g->nx + 2 * g->nb;
    p->pitch = (p->NX + 31) / 32 * 32;
    p->S = sh->S;
    p->field = (long long)p->NZ * p->pitch;
    const int S = sh->S;
    p->nt.assign(sh->nt, sh->nt + S);
    p->nt_max = *std::max_element(p->nt.begin(), p->nt.end());
    // tiles
    const int TZ = o.tile_z ? o.tile_z : TZ_DEFAULT;
    const int ntz = (p->NZ + TZ - 1) / TZ, ntx = (p->pitch + TX - 1) / TX, ntiles = ntz * ntx;
    // sources, receivers, per-tile receiver lists, trace offsets
    std::vector<int> src_pt(S), nrec(S);
    std::vector<std::vector<std::pair<int, int>>> per_tile((size_t)S * ntiles);
    p->tr_off.resize(S);
    long long off = 0;
    for (int s = 0; s < S; ++s) {
        if (sh->src_iz[s] < 0 || sh->src_iz[s] >= g->nz || sh->src_ix[s] < 0 || sh->src_ix[s] >= g->nx) {
            delete p;
            return fail(nullptr, AAFWI_ERR_OOB, "source outside the physical grid");
        }
        src_pt[s] = (sh->src_iz[s] + g->nb) * p->pitch + sh->src_ix[s] + g->nb;
        const int r0 = sh->rec_off[s], r1 = sh->rec_off[s + 1];
        if (r1 < r0) {
            delete p;
            return fail(nullptr, AAFWI_ERR_ARG, "rec_off must be non-decreasing");
        }
        nrec[s] = r1 - r0;
        std::set<int> seen;
        for (int j = 0; j < nrec[s]; ++j) {
            const int iz = sh->rec_iz[r0 + j], ix = sh->rec_ix[r0 + j];
            if (iz < 0 || iz >= g->nz || ix < 0 || ix >= g->nx) {
                delete p;
                return fail(nullptr, AAFWI_ERR_OOB, "receiver outside the physical grid");
            }
            const int pz = iz + g->nb, px = ix + g->nb;
            const int pt = pz * p->pitch + px;
            if (!seen.insert(pt).second) {
                delete p;
                return fail(nullptr, AAFWI_ERR_ARG, "duplicate receiver cell within a shot");
            }
            per_tile[(size_t)s * ntiles + (pz / TZ) * ntx + px / TX].push_back({pt, j});
        }
        p->tr_off[s] = off;
        off += (long long)p->nt[s] * nrec[s];
    }
    p->trace_count = off;
    std::vector<int> trec_off(1, 0), trec_pt, trec_col;
    for (auto &v : per_tile) {
        for (auto &e : v) {
            trec_pt.push_back(e.first);
            trec_col.push_back(e.second);
        }
        trec_off.push_back((int)trec_pt.size());
    }
    // sponge tables 1 - g(d) (FP64 -> FP32; 1 beyond NX so that G = 0 in the
    // pitch padding) and the wavelet in stencil units 5040 dx^2 w(t_n)/(dx dz)
    auto depth = [&](int i, int n) { return i < g->nb ? g->nb - i : (i > n - 1 - g->nb ? i - (n - 1 - g->nb) : 0); };
    std::vector<float> dGz(p->NZ), dGx(p->pitch, 1.f), ws(p->nt_max);
    for (int i = 0; i < p->NZ; ++i) dGz[i] = (float)(1.0 - std::exp(-std::pow(kSpongeA * depth(i, p->NZ), 2)));
    for (int i = 0; i < p->NX; ++i) dGx[i] = (float)(1.0 - std::exp(-std::pow(kSpongeA * depth(i, p->NX), 2)));
    const double t5040 = 5040.0 * g->dx * g->dx;
    for (int n = 0; n < p->nt_max; ++n) ws[n] = (float)(t5040 * wavelet[n] / (g->dx * g->dz));
    // workspace plan
    const PlanLayout lay = plan_layout(p->field, (long long)p->NZ * p->NX, S, p->nt_max, p->trace_count, o);
    p->Sb = lay.Sb;
    p->nbatch = lay.nbatch;
    p->full = lay.full;
    p->k = lay.k;
    p->nck = lay.nck;
    p->ws_bytes = lay.bytes;
    const size_t budget = lay.budget;
    if (!lay.fits) {
        char b[200];
        snprintf(b, sizeof b, "workspace %.2f GB exceeds the budget %.2f GB", p->ws_bytes / 1e9, budget / 1e9);
        delete p;
        return fail(nullptr, AAFWI_ERR_NOMEM, b);
    }
    // device allocations
    int *d_nt, *d_src, *d_toff, *d_tpt, *d_tcol, *d_nrec;
    float *d_ws, *d_Gz, *d_Gx;  // wavelet, 1 - g tables
    long long *d_troff;
    std::vector<int> trec_pt_nz = trec_pt.empty() ? std::vector<int>{0} : trec_pt;
    std::vector<int> trec_col_nz = trec_col.empty() ? std::vector<int>{0} : trec_col;
    bool ok = upload(p->bufs, &d_nt, p->nt) && upload(p->bufs, &d_src, src_pt) &&
              upload(p->bufs, &d_toff, trec_off) && upload(p->bufs, &d_tpt, trec_pt_nz) &&
              upload(p->bufs, &d_tcol, trec_col_nz) && upload(p->bufs, &d_nrec, nrec) &&
              upload(p->bufs, &d_ws, ws) && upload(p->bufs, &d_Gz, dGz) && upload(p->bufs, &d_Gx, dGx) &&
              upload(p->bufs, &d_troff, p->tr_off);
    const long long ps = (long long)p->Sb * p->field;   // one slot: the batch's shots
    ok = ok && dalloc(p->bufs, &p->W, 2 * p->field) && dalloc(p->bufs, &p->rho_pad, p->field) &&
         dalloc(p->bufs, &p->dbuf, 2 * ps) && dalloc(p->bufs, &p->zbuf, 2 * ps) && dalloc(p->bufs, &p->fbuf, 4 * ps) &&
         dalloc(p->bufs, &p->img, ps) && dalloc(p->bufs, &p->dsyn, p->trace_count) &&
         dalloc(p->bufs, &p->resid, p->trace_count) && dalloc(p->bufs, &p->partials, RED_BLOCKS) &&
         dalloc(p->bufs, &p->J, 1) && dalloc(p->bufs, &p->err, 1) &&
         dalloc(p->bufs, &p->rowsum, (size_t)p->NZ * p->nx);
    if (ok) {
        if (p->full) {
            ok = dalloc(p->bufs, &p->hist, (p->nt_max + 1) * ps);
        } else {
            ok = dalloc(p->bufs, &p->hist, 2LL * p->nck * ps) && dalloc(p->bufs, &p->rbuf, (long long)p->k * ps);
        }
    }
    if (!ok) {
        free_bufs(p->bufs);
        delete p;
        return fail(nullptr, AAFWI_ERR_NOMEM, "cudaMalloc failed for the plan workspace");
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_bufs(p->bufs);
        delete p;
        return cuda_fail(nullptr, e, "plan initialisation");
    }
    Geo &G = p->geo;
    G.NZ = p->NZ; G.NX = p->NX; G.pitch = p->pitch; G.nb = p->nb; G.S = p->Sb; G.shot0 = 0;
    G.tz = TZ; G.ntz = ntz; G.ntx = ntx; G.ntiles = ntiles; G.field = p->field;
    G.err = p->err;
    G.rz = (float)((g->dx * g->dx) / (g->dz * g->dz));
    p->K = g->dt * g->dt / t5040;
    G.iscale = (float)(-1.0 / (g->dt * g->dt));
    G.tscale = (float)(1.0 / t5040);
    G.inj_scale = (float)t5040;
    G.nt = d_nt; G.src_pt = d_src; G.ws = d_ws; G.dGz = d_Gz; G.dGx = d_Gx;
    G.nt_min = *std::min_element(p->nt.begin(), p->nt.end());
    G.trec_off = d_toff; G.trec_pt = d_tpt; G.trec_col = d_tcol; G.tr_off = d_troff; G.nrec = d_nrec;
    {
        std::string why;
        auto map = [&](CUtensorMap *m, const float *buf, int slots, bool halo) {
            return encode_tile_map(m, buf, p->NX, p->NZ, p->pitch, p->field, p->Sb, slots, TZ, halo ? HALO : 0,
                                   &why);
        };
        bool mk = map(&p->tm_f, p->fbuf, 4, true) && map(&p->tm_fi, p->fbuf, 4, false) &&
                  encode_tile_map(&p->tm_f8, p->fbuf, p->NX, p->NZ, p->pitch, p->field, p->Sb, 4, TZ, 2 * HALO,
                                  &why) &&
                  map(&p->tm_d, p->dbuf, 2, true) && map(&p->tm_di, p->dbuf, 2, false) &&
                  encode_tile_map(&p->tm_rho, p->rho_pad, p->NX, p->NZ, p->pitch, p->field, 1, 1, TZ, 0, &why) &&
                  map(&p->tm_z, p->zbuf, 2, true) &&
                  map(&p->tm_zi, p->zbuf, 2, false) &&
                  encode_tile_map(&p->tm_w, p->W, p->NX, p->NZ, p->pitch, p->field, 1, 2, TZ, 0, &why);
        if (mk && p->full) mk = map(&p->tm_t, p->hist, p->nt_max + 1, false);
        if (mk && !p->full)
            mk = map(&p->tm_ck, p->hist, 2 * p->nck, true) && map(&p->tm_cki, p->hist, 2 * p->nck, false) &&
                 map(&p->tm_t, p->rbuf, p->k, false);
        if (!mk) {
            free_bufs(p->bufs);
            delete p;
            return fail(nullptr, AAFWI_ERR_CUDA, "tile descriptors: " + why);
        }
    }
    {
        std::string why;
        const int rc = setup_persist(p, o.engine, sh, &why);
        if (rc) {
            free_bufs(p->bufs);
            delete p;
            return fail(nullptr, rc, why);
        }
    }
    *out = p;
    return AAFWI_OK;
}

void aafwi_plan_destroy(aafwi_plan *p)
{
    if (!p) return;
    drop_graphs(p);
    free_bufs(p->bufs);
    delete p;
}

int aafwi_plan_set_stall(aafwi_plan *p, int step)
{
    if (!p) return AAFWI_ERR_ARG;
    if (!p->persist_adj && step >= 0) return fail(p, AAFWI_ERR_STATE, "plan has no persistent sweeps");
    p->stall_step = step < 0 ? -1 : step;
    return AAFWI_OK;
}

int aafwi_plan_get_info(const aafwi_plan *p, aafwi_plan_info *info)
{
    if (!p || !info) return AAFWI_ERR_ARG;
    info->NZ = p->NZ; info->NX = p->NX; info->pitch = p->pitch;
    info->S = p->S; info->nt_max = p->nt_max;
    info->trace_count = p->trace_count;
    info->checkpoint_every = p->k;
    info->n_checkpoints = p->nck;
    info->workspace_bytes = p->ws_bytes;
    info->tile_z = p->geo.tz; info->tile_x = TX;
    info->n_tiles = p->geo.ntiles;
    info->engine = p->persist_fwd ? AAFWI_ENGINE_PERSISTENT
                   : p->persist_adj ? AAFWI_ENGINE_HYBRID : AAFWI_ENGINE_PER_STEP;
    info->persist_ctas = p->persist_adj ? p->pgeo.P : 0;
    info->shots_per_batch = p->Sb;
    info->n_batches = p->nbatch;
    info->steps_per_launch = (p->full && p->steps_per_launch == 2 && !p->persist_fwd) ? 2 : 1;
    info->lanes = std::min(p->lanes, p->Sb);
    return AAFWI_OK;
}

int aafwi_model_forward(aafwi_plan *p, const float *m, float *d_out, aafwi_stream stream)
{
    if (int rc0 = refuse_retired(p)) return rc0;
    if (!p || !m) return fail(p, AAFWI_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    p->fwd_valid = false;
    if ((rc = prep(p, m, nullptr, st))) return rc;
    // with several batches only the last batch's wavefield would survive, and
    // no adjoint can reuse it: store no history
    for (int b = 0; b < p->nbatch; ++b)
        if ((rc = run_forward(p, b, false, p->dsyn, st, p->nbatch == 1))) return rc;
    if (d_out && d_out != p->dsyn &&
        cudaMemcpyAsync(d_out, p->dsyn, p->trace_count * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return cuda_fail(p, cudaGetLastError(), "copy traces");
    p->fwd_valid = p->nbatch == 1;   // with batches only the last batch's wavefield is kept
    p->fwd_model = m;
    return AAFWI_OK;
}

int aafwi_born_forward(aafwi_plan *p, const float *m0, const float *rho, float *d_out, aafwi_stream stream)
{
    if (int rc0 = refuse_retired(p)) return rc0;
    if (!p || !m0 || !rho || !d_out) return fail(p, AAFWI_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    p->fwd_valid = false;
    if ((rc = prep(p, m0, rho, st))) return rc;
    for (int b = 0; b < p->nbatch; ++b)
        if ((rc = run_forward(p, b, true, d_out, st))) return rc;
    return AAFWI_OK;
}

int aafwi_misfit(aafwi_plan *p, const float *d_syn, const float *d_obs, float *resid, double *J_host,
                 aafwi_stream stream)
{
    if (int rc0 = refuse_retired(p)) return rc0;
    if (!p || !d_syn || !d_obs) return fail(p, AAFWI_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    launch_misfit(d_syn, d_obs, resid, p->trace_count, p->partials, p->J, st);
    int rc = check_launch(p);
    if (rc) return rc;
    return finish_sync(p, J_host, st);
}

int aafwi_read_misfit(aafwi_plan *p, double *J_host, aafwi_stream stream)
{
    if (int rc0 = refuse_retired(p)) return rc0;
    if (!p || !J_host) return fail(p, AAFWI_ERR_ARG, "NULL argument");
    return finish_sync(p, J_host, (cudaStream_t)stream);
}

namespace {

// CSR trace range [first, first + count) of batch b.
void batch_traces(const aafwi_plan *p, int b, long long *first, long long *count)
{
    const int s0 = b * p->Sb, s1 = std::min(p->S, s0 + p->Sb);
    *first = p->tr_off[s0];
    *count = (s1 < p->S ? p->tr_off[s1] : p->trace_count) - *first;
}

// Adjoint sweeps of every batch (the forward of each batch first -- the Born
// pair when fwd_born -- unless the stored one is reused), imaging (Born scale
// when adj_born), shot sum and E^T into out.  With d_obs the adjoint source is
// the residual d_syn - d_obs of each batch (and J is formed over all traces),
// else adj_src.
int gradient_pass(aafwi_plan *p, bool fwd_born, bool adj_born, bool reuse, const float *d_obs, const float *adj_src,
                  float *out, cudaStream_t st)
{
    int rc;
    for (int b = 0; b < p->nbatch; ++b) {
        if (!reuse && (rc = run_forward(p, b, fwd_born, d_obs ? p->dsyn : nullptr, st))) return rc;
        const float *r = adj_src;
        if (d_obs) {
            if (p->nbatch == 1) {
                launch_misfit(p->dsyn, d_obs, p->resid, p->trace_count, p->partials, p->J, st);
            } else {
                long long first, count;
                batch_traces(p, b, &first, &count);
                launch_misfit(p->dsyn + first, d_obs + first, p->resid + first, count, p->partials, p->J, st);
            }
            r = p->resid;
        }
        if ((rc = run_adjoint(p, b, adj_born, r, st))) return rc;
        launch_shot_sum(batch_geo(p, b), p->nz, p->nx, p->img, p->rowsum, b > 0,
                        b + 1 == p->nbatch ? out : nullptr, st);
    }
    if (d_obs && p->nbatch > 1)   // J over all traces, in the same order as without batches
        launch_misfit(p->dsyn, d_obs, nullptr, p->trace_count, p->partials, p->J, st);
    return check_launch(p);
}

}  // namespace

int aafwi_adjoint_gradient(aafwi_plan *p, int mode, const float *m, const float *rho, const float *d_obs,
                           float *grad, double *J_host, int flags, aafwi_stream stream)
{
    if (int rc0 = refuse_retired(p)) return rc0;
    if (!p || !m || !d_obs || !grad) return fail(p, AAFWI_ERR_ARG, "NULL argument");
    if (mode != AAFWI_MODE_FWI && mode != AAFWI_MODE_LSRTM) return fail(p, AAFWI_ERR_ARG, "unknown mode");
    if (mode == AAFWI_MODE_LSRTM && !rho) return fail(p, AAFWI_ERR_ARG, "LSRTM needs rho");
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    const bool born = mode == AAFWI_MODE_LSRTM;
    const bool reuse = !born && (flags & AAFWI_REUSE_FORWARD);
    if (reuse) {
        if (!p->fwd_valid || p->fwd_model != m)
            return fail(p, AAFWI_ERR_STATE, "no stored forward wavefield for this model");
    } else {
        p->fwd_valid = false;
        if ((rc = prep(p, m, born ? rho : nullptr, st))) return rc;
    }
    if ((rc = gradient_pass(p, born, born, reuse, d_obs, nullptr, grad, st))) return rc;
    if (!born) {
        p->fwd_valid = p->nbatch == 1;
        p->fwd_model = m;
    }
    return finish_sync(p, J_host, st);
}

int aafwi_adjoint_gradient_host(aafwi_plan *p, int mode, const float *m, const float *rho, const float *d_obs,
                                float *grad, double *J_host, aafwi_stream stream)
{
    if (int rc0 = refuse_retired(p)) return rc0;
    if (!p || !m || !d_obs || !grad || !J_host) return fail(p, AAFWI_ERR_ARG, "NULL argument");
    if (mode != AAFWI_MODE_FWI && mode != AAFWI_MODE_LSRTM) return fail(p, AAFWI_ERR_ARG, "unknown mode");
    if (mode == AAFWI_MODE_LSRTM && !rho) return fail(p, AAFWI_ERR_ARG, "LSRTM needs rho");
    const size_t n = (size_t)p->nz * p->nx;
    bool ok = (p->stage_m || dalloc(p->bufs, &p->stage_m, n)) && (p->stage_rho || dalloc(p->bufs, &p->stage_rho, n)) &&
              (p->stage_d || dalloc(p->bufs, &p->stage_d, (size_t)p->trace_count)) &&
              (p->stage_g || dalloc(p->bufs, &p->stage_g, n));
    if (!ok) return fail(p, AAFWI_ERR_NOMEM, "device staging buffers for host arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const bool born = mode == AAFWI_MODE_LSRTM;
    cudaError_t e = cudaMemcpyAsync(p->stage_m, m, n * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && born) e = cudaMemcpyAsync(p->stage_rho, rho, n * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->stage_d, d_obs, (size_t)p->trace_count * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(p, e, "host to device copy");
    const int rc = aafwi_adjoint_gradient(p, mode, p->stage_m, born ? p->stage_rho : nullptr, p->stage_d, p->stage_g,
                                          nullptr, 0, stream);
    if (rc) return rc;
    e = cudaMemcpyAsync(grad, p->stage_g, n * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(p, e, "device to host copy");
    return finish_sync(p, J_host, st);
}

int aafwi_fwi_adjoint(aafwi_plan *p, const float *m, const float *adj_src, float *grad, int flags,
                      aafwi_stream stream)
{
    if (int rc0 = refuse_retired(p)) return rc0;
    if (!p || !m || !adj_src || !grad) return fail(p, AAFWI_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    const bool reuse = flags & AAFWI_REUSE_FORWARD;
    if (reuse) {
        if (!p->fwd_valid || p->fwd_model != m)
            return fail(p, AAFWI_ERR_STATE, "no stored forward wavefield for this model");
    } else {
        p->fwd_valid = false;
        if ((rc = prep(p, m, nullptr, st))) return rc;
    }
    if ((rc = gradient_pass(p, false, false, reuse, nullptr, adj_src, grad, st))) return rc;
    p->fwd_valid = p->nbatch == 1;
    p->fwd_model = m;
    return AAFWI_OK;
}

int aafwi_born_adjoint(aafwi_plan *p, const float *m0, const float *resid, float *img, aafwi_stream stream)
{
    if (int rc0 = refuse_retired(p)) return rc0;
    if (!p || !m0 || !resid || !img) return fail(p, AAFWI_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    p->fwd_valid = false;
    if ((rc = prep(p, m0, nullptr, st))) return rc;
    return gradient_pass(p, false, true, false, nullptr, resid, img, st);
}

// ---------------------------------------------------------------------------
// Anderson acceleration
// ---------------------------------------------------------------------------

int aafwi_aa_create(size_t n, int M, double eta, aafwi_aa **out)
{
    if (!out || n == 0 || M < 0 || M > AA_MAXM)
        return fail(nullptr, AAFWI_ERR_ARG, "aa_create: need n > 0 and 0 <= M <= 20");
    *out = nullptr;
    auto *a = new aafwi_aa();
    cudaGetDevice(&a->device);
    AAState &s = a->s;
    s.n = (long long)n;
    s.M = M;
    s.eta = eta;
    s.beta = 1.0;
    s.norm = AAFWI_NORM_L2;
    const int M1 = M + 1;
    bool ok = dalloc(a->bufs, &s.ring_p, (size_t)M1 * n) && dalloc(a->bufs, &s.ring_g, (size_t)M1 * n) &&
              dalloc(a->bufs, &s.gram, (size_t)M1 * M1) &&
              dalloc(a->bufs, &s.partials, (size_t)RED_BLOCKS * (2 * AA_MAXM)) &&
              dalloc(a->bufs, &s.gamma, AA_MAXM) && dalloc(a->bufs, &s.meta, 4) && dalloc(a->bufs, &s.dot, 1);
    if (!ok) {
        free_bufs(a->bufs);
        delete a;
        return fail(nullptr, AAFWI_ERR_NOMEM, "cudaMalloc failed for the AA state");
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        free_bufs(a->bufs);
        delete a;
        return fail(nullptr, AAFWI_ERR_CUDA, "aa_create initialisation");
    }
    *out = a;
    return AAFWI_OK;
}

void aafwi_aa_destroy(aafwi_aa *a)
{
    if (!a) return;
    free_bufs(a->bufs);
    delete a;
}

int aafwi_aa_set_eta(aafwi_aa *a, double eta)
{
    if (!a || !(eta > 0)) return AAFWI_ERR_ARG;
    a->s.eta = eta;
    return AAFWI_OK;
}

int aafwi_aa_set_weights(aafwi_aa *a, const float *w, aafwi_stream stream)
{
    if (!a) return AAFWI_ERR_ARG;
    if (a->s.count > 0) return fail(nullptr, AAFWI_ERR_STATE, "aa_set_weights after the first aa_step");
    cudaStream_t st = (cudaStream_t)stream;
    if (!w) {
        a->s.weights = nullptr;
        return AAFWI_OK;
    }
    if (!a->wbuf && !dalloc(a->bufs, &a->wbuf, (size_t)a->s.n))
        return fail(nullptr, AAFWI_ERR_NOMEM, "cudaMalloc failed for the AA weights");
    cudaError_t e = cudaMemcpyAsync(a->wbuf, w, (size_t)a->s.n * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "aa_set_weights copy");
    a->s.weights = a->wbuf;
    return AAFWI_OK;
}

int aafwi_aa_set_beta(aafwi_aa *a, double beta)
{
    if (!a || !(beta >= 0.0) || beta > 1.0) return AAFWI_ERR_ARG;
    a->s.beta = beta;
    return AAFWI_OK;
}

int aafwi_aa_set_norm(aafwi_aa *a, int norm)
{
    if (!a || (norm != AAFWI_NORM_L2 && norm != AAFWI_NORM_L1 && norm != AAFWI_NORM_LINF))
        return fail(nullptr, AAFWI_ERR_ARG, "aa_set_norm: unknown norm");
    AAState &s = a->s;
    if (norm != AAFWI_NORM_L2 && !s.lp_rows) {
        const bool ok = dalloc(a->bufs, &s.lp_rows, AA_LP_ROWS) && dalloc(a->bufs, &s.lp_cnt, 1) &&
                        dalloc(a->bufs, &s.lp_part, (size_t)RED_BLOCKS * (AA_MAXM + 1)) &&
                        dalloc(a->bufs, &s.lp_gat, (size_t)AA_LP_ROWS * (AA_MAXM + 2));
        if (!ok) return fail(nullptr, AAFWI_ERR_NOMEM, "cudaMalloc failed for the l1 / l-infinity buffers");
    }
    s.norm = norm;
    return AAFWI_OK;
}

int aafwi_aa_get_lp_info(const aafwi_aa *a, aafwi_aa_lp_info *info)
{
    if (!a || !info) return AAFWI_ERR_ARG;
    info->objective = a->s.lp.objective;
    info->lower_bound = a->s.lp.lower_bound;
    info->rounds = a->s.lp.rounds;
    info->rows = a->s.lp.rows;
    return AAFWI_OK;
}

int aafwi_aa_step(aafwi_aa *a, const float *p_k, const float *grad_k, float *p_tilde, float *p_bar,
                  double *gamma_host, int *Mk_host, aafwi_stream stream)
{
    if (!a || !p_k || !grad_k || !p_tilde || !p_bar) return fail(nullptr, AAFWI_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    AAState &s = a->s;
    launch_aa_step(s, p_k, grad_k, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "aa_step launch");
    if (s.norm != AAFWI_NORM_L2 && s.count > 1) {
        // l1 / l-infinity: the LP rounds start from the l2 solution over the
        // columns its rank safeguard keeps
        int meta[2] = {0, 0};
        double gl2[AA_MAXM], glp[AA_MAXM];
        e = cudaMemcpyAsync(meta, s.meta, sizeof meta, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(gl2, s.gamma, sizeof gl2, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "aa_step readback");
        if (meta[0] > 0) {
            std::string msg;
            const int rc = aa_lp_gamma(s, s.slots + meta[1], meta[0], s.norm, gl2, glp, &s.lp, &msg, st);
            if (rc) return fail(nullptr, rc, rc == AAFWI_ERR_CUDA ? std::string("aa_step: l1 / l-infinity pass failed")
                                                                : msg);
            e = cudaMemcpyAsync(s.gamma, glp, meta[0] * sizeof(double), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // glp lives on this stack frame
            if (e != cudaSuccess) return cuda_fail(nullptr, e, "aa_step gamma upload");
        }
    }
    launch_aa_mix(s, p_tilde, p_bar, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "aa_step launch");
    if (gamma_host || Mk_host) {
        int meta[2] = {0, 0};
        double gam[AA_MAXM];
        e = cudaMemcpyAsync(meta, s.meta, sizeof meta, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(gam, s.gamma, sizeof gam, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "aa_step readback");
        if (Mk_host) *Mk_host = meta[0];
        if (gamma_host)
            for (int j = 0; j < s.M; ++j) gamma_host[j] = j < meta[0] ? gam[j] : 0.0;
    }
    return AAFWI_OK;
}

int aafwi_aa_combine(aafwi_aa *a, double lambda, const float *p_tilde, const float *p_bar, float *p_next,
                     float lo, float hi, double *armijo_dot_host, aafwi_stream stream)
{
    if (!a || !p_tilde || !p_bar || !p_next) return fail(nullptr, AAFWI_ERR_ARG, "NULL argument");
    if (a->s.count == 0) return fail(nullptr, AAFWI_ERR_STATE, "aa_combine before aa_step");
    cudaStream_t st = (cudaStream_t)stream;
    launch_aa_combine(a->s, (float)lambda, p_tilde, p_bar, p_next, lo, hi, armijo_dot_host != nullptr, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "aa_combine launch");
    if (armijo_dot_host) {
        e = cudaMemcpyAsync(armijo_dot_host, a->s.dot, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "aa_combine readback");
    }
    return AAFWI_OK;
}

int aafwi_absmax(const float *x, size_t n, double *host_out, aafwi_stream stream)
{
    if (!x || !host_out || n == 0) return fail(nullptr, AAFWI_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_red_mu);
    double *buf = nullptr;
    if (!reduction_scratch(&buf)) return fail(nullptr, AAFWI_ERR_NOMEM, "absmax scratch");
    launch_absmax(x, (long long)n, buf, buf + RED_BLOCKS, st);
    cudaError_t e = cudaMemcpyAsync(host_out, buf + RED_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "absmax");
    return AAFWI_OK;
}

int aafwi_dot(const float *x, const float *y, size_t n, double *host_out, aafwi_stream stream)
{
    if (!x || !y || !host_out || n == 0) return fail(nullptr, AAFWI_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_red_mu);
    double *buf = nullptr;
    if (!reduction_scratch(&buf)) return fail(nullptr, AAFWI_ERR_NOMEM, "dot scratch");
    launch_dot(x, y, (long long)n, buf, buf + RED_BLOCKS, st);
    cudaError_t e = cudaMemcpyAsync(host_out, buf + RED_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "dot");
    return AAFWI_OK;
}

int aafwi_axpby(double a, const float *x, double b, float *y, size_t n, aafwi_stream stream)
{
    if (!x || !y || n == 0) return fail(nullptr, AAFWI_ERR_ARG, "NULL argument");
    launch_axpby((float)a, x, (float)b, y, (long long)n, (cudaStream_t)stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "axpby");
    return AAFWI_OK;
}

int aafwi_axpby_clip(double a, const float *x, double b, float *y, size_t n, float lo, float hi, aafwi_stream stream)
{
    if (!x || !y || n == 0) return fail(nullptr, AAFWI_ERR_ARG, "NULL argument");
    launch_axpby((float)a, x, (float)b, y, (long long)n, (cudaStream_t)stream, lo, hi);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "axpby_clip");
    return AAFWI_OK;
}

unsigned long long aafwi_launch_count(void)
{
    return g_launch_count.load(std::memory_order_relaxed);
}

}  // extern "C"
