// autotune.cu -- choice of the sweeps' launch configuration (engine: per
// step, persistent or hybrid; tile height and shot lanes of the per-step
// kernels) by timing short sweeps of temporary plans of the same geometry.
// Host code over the public entry points only.
#include <algorithm>
#include <vector>

#include "internal.cuh"

using namespace aafwi;

namespace {

struct Candidate {
    int engine, tile_z, lanes;   // lanes 0: the plan default
};

struct Scratch {
    float *d_obs = nullptr, *grad = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Scratch()
    {
        if (d_obs) cudaFree(d_obs);
        if (grad) cudaFree(grad);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
    }
};

int tune_fail(int code, const char *msg)
{
    set_call_error(msg);
    return code;
}

// Median time of `reps` (forward sweep + adjoint sweep reusing it) on plan p.
int time_plan(aafwi_plan *p, const float *m, Scratch &sc, int reps, double *ms)
{
    double J = 0.0;
    int rc = aafwi_adjoint_gradient(p, AAFWI_MODE_FWI, m, nullptr, sc.d_obs, sc.grad, &J, 0, sc.st);   // warm-up
    if (rc) return rc;
    std::vector<double> t;
    for (int r = 0; r < reps; ++r) {
        if (cudaEventRecord(sc.e0, sc.st) != cudaSuccess) return AAFWI_ERR_CUDA;
        if ((rc = aafwi_model_forward(p, m, nullptr, sc.st))) return rc;
        if ((rc = aafwi_adjoint_gradient(p, AAFWI_MODE_FWI, m, nullptr, sc.d_obs, sc.grad, nullptr,
                                         AAFWI_REUSE_FORWARD, sc.st)))
            return rc;
        if (cudaEventRecord(sc.e1, sc.st) != cudaSuccess || cudaEventSynchronize(sc.e1) != cudaSuccess)
            return AAFWI_ERR_CUDA;
        float f = 0.f;
        cudaEventElapsedTime(&f, sc.e0, sc.e1);
        t.push_back(f);
    }
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return aafwi_read_misfit(p, &J, sc.st);   // surfaces a NaN / CFL flag raised by the runs
}

}  // namespace

extern "C" int aafwi_autotune(const aafwi_grid *grid, const aafwi_shots *shots, const double *wavelet,
                              const float *m, int steps, int reps, const aafwi_plan_opts *base,
                              aafwi_tune_entry *table, int table_cap, int *n_entries, aafwi_plan_opts *best)
{
    if (!grid || !shots || !wavelet || !m || !best || steps < 1 || reps < 1 || table_cap < 0 ||
        (table_cap > 0 && !table) || !shots->nt || shots->S < 1 || !shots->rec_off)
        return tune_fail(AAFWI_ERR_ARG, "autotune: invalid argument");
    aafwi_plan_opts o{};
    if (base) o = *base;
    const int S = shots->S;
    // would a plan of the full record keep the full history?
    const int NZ = grid->nz + 2 * grid->nb, pitch = (grid->nx + 2 * grid->nb + 31) / 32 * 32;
    int nt_max = 0;
    long long traces = 0;
    std::vector<int> nt(shots->nt, shots->nt + S);
    for (int s = 0; s < S; ++s) {
        nt_max = std::max(nt_max, nt[s]);
        traces += (long long)nt[s] * (shots->rec_off[s + 1] - shots->rec_off[s]);
        nt[s] = std::min(nt[s], steps);
    }
    const int NX = grid->nx + 2 * grid->nb;
    const PlanLayout lay = plan_layout((long long)NZ * pitch, (long long)NZ * NX, S, nt_max, traces, o);
    const bool full = lay.full && lay.nbatch == 1;   // what the persistent engines need
    std::vector<Candidate> cands;
    auto allowed = [&](int e) { return o.engine == AAFWI_ENGINE_AUTO || o.engine == e; };
    if (allowed(AAFWI_ENGINE_PER_STEP))
        for (int tz : {16, 32, 64}) cands.push_back({AAFWI_ENGINE_PER_STEP, tz, o.lanes});
    if (full && allowed(AAFWI_ENGINE_PERSISTENT)) cands.push_back({AAFWI_ENGINE_PERSISTENT, 0, o.lanes});
    if (full && allowed(AAFWI_ENGINE_HYBRID))
        for (int tz : {16, 32, 64}) cands.push_back({AAFWI_ENGINE_HYBRID, tz, o.lanes});
    if (cands.empty())
        return tune_fail(AAFWI_ERR_ARG, "autotune: the persistent engines need the full history of all shots at once");
    // A plan of the full record that runs its shots in batches sweeps one
    // batch at a time: time the candidates on one batch (the first lay.Sb
    // shots) so that a launch covers the shots it will cover in that plan.
    aafwi_shots sh = *shots;
    sh.nt = nt.data();
    if (lay.nbatch > 1) sh.S = lay.Sb;
    Scratch sc;
    if (cudaStreamCreateWithFlags(&sc.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&sc.e0) != cudaSuccess || cudaEventCreate(&sc.e1) != cudaSuccess)
        return tune_fail(AAFWI_ERR_CUDA, "autotune: stream / events");
    int ntimed = 0;
    double best_ms = -1.0;
    Candidate win{};
    // one candidate: a temporary plan timed on the cut records; false if it
    // does not qualify (persistent strips), rc set on an error
    auto try_one = [&](const Candidate &c, int *rc) -> bool {
        aafwi_plan_opts co = o;
        co.engine = c.engine;
        co.tile_z = c.tile_z;
        co.lanes = c.lanes;
        co.checkpoint_every = 1;
        aafwi_plan *p = nullptr;
        *rc = aafwi_plan_create(grid, &sh, wavelet, &co, &p);
        if (*rc == AAFWI_ERR_ARG && c.engine != AAFWI_ENGINE_PER_STEP) {   // strips do not qualify
            *rc = AAFWI_OK;
            return false;
        }
        if (*rc) return false;
        aafwi_plan_info info{};
        aafwi_plan_get_info(p, &info);
        if (!sc.d_obs) {
            const size_t nt_bytes = std::max<long long>(info.trace_count, 1) * sizeof(float);
            if (cudaMalloc(&sc.d_obs, nt_bytes) != cudaSuccess ||
                cudaMalloc(&sc.grad, (size_t)grid->nz * grid->nx * sizeof(float)) != cudaSuccess ||
                cudaMemset(sc.d_obs, 0, nt_bytes) != cudaSuccess) {
                cudaGetLastError();
                aafwi_plan_destroy(p);
                *rc = tune_fail(AAFWI_ERR_NOMEM, "autotune: scratch buffers");
                return false;
            }
        }
        double ms = 0.0;
        *rc = time_plan(p, m, sc, reps, &ms);
        if (*rc) {
            set_call_error(aafwi_last_error(p));
            aafwi_plan_destroy(p);
            return false;
        }
        aafwi_plan_destroy(p);
        if (ntimed < table_cap) table[ntimed] = {c.engine, c.tile_z, info.lanes, ms};
        ++ntimed;
        if (best_ms < 0 || ms < best_ms) {
            best_ms = ms;
            win = c;
        }
        return true;
    };
    for (const Candidate &c : cands) {
        int rc = AAFWI_OK;
        try_one(c, &rc);
        if (rc) return rc;
    }
    // shot lanes of the winner's per-step sweeps (more than the shots: the same plan)
    if (ntimed > 0 && o.lanes == 0 && win.engine != AAFWI_ENGINE_PERSISTENT) {
        const Candidate w = win;
        for (int l : {1, 2, 8}) {
            if (l > sh.S) continue;
            int rc = AAFWI_OK;
            try_one({w.engine, w.tile_z, l}, &rc);
            if (rc) return rc;
        }
    }
    if (n_entries) *n_entries = ntimed;
    if (ntimed == 0) return tune_fail(AAFWI_ERR_ARG, "autotune: no configuration qualifies");
    *best = o;
    best->engine = win.engine;
    best->tile_z = win.tile_z;
    best->lanes = win.lanes;
    return AAFWI_OK;
}
