// wave_kernels.cu -- time-step kernels of the 2D constant-density acoustic
// wave equation (Sec. 2.2, eq. FWD), its Born linearisation (eq. Born) and
// its exact discrete adjoint fused with the imaging condition (eqs. FWI_adj,
// adj_grad1).
//
// Scheme (leap-frog, 8th-order Laplacian L, Cerjan sponge G, W = dt^2/m):
//   forward   u^{n+1} = G (2 u^n - G u^{n-1} + W (L u^n + s^n))
//   Born      du^{n+1} = G (2 du^n - G du^{n-1} + W L du^n) - G W rho (L u^n + s^n)
//   adjoint   z^n = G (2 z^{n+1} - G z^{n+2} + W (L z^{n+1} + R^T r^n))
//   imaging   img += scale z^n (L u^n + s^n),  scale = -1/m (FWI) or -1 (Born)
// The forward (and Born) step can store T^n = 5040 dx^2 (L u^n + s^n), the
// stencil result it computes anyway; the adjoint step reads T^n back for the
// imaging condition, so it stages only z^{n+1} and evaluates one stencil.
//
// FP32 evaluation (stencil_math.cuh, shared with the persistent kernels)
// keeps the rounding error of long runs small, since the residual of an
// inversion is often < 1 % of the data and trace errors are amplified in the
// misfit and the gradient: L as differences to the centre cell with integer
// weights, W as the FP64-derived pair Wh + Wl, G x as x - (1 - G) x; every
// rounding explicit, pairs of cells on packed FP32x2 instructions.
//
// One launch advances every shot of a lane (a set of consecutive shots of
// the batch) by one step: grid (x tiles, z tiles, shots of the lane).
// A CTA stages its tz x TX tile plus a 4-cell halo of each stencil input in
// shared memory with 128-bit loads; each thread owns one float4 column group
// on tz/8 rows.  Source injection, receiver gather and residual injection are
// fused into the same launch through a per-(shot, tile) receiver list.
#include <cudaTypedefs.h>   // PFN_cuTensorMapEncodeTiled

#include "internal.cuh"
#include "stencil_math.cuh"

namespace aafwi {

std::atomic<unsigned long long> g_launch_count{0};
thread_local unsigned long long *g_capture_count = nullptr;


typedef float Tile[SW];
typedef float Tile8[SW8];   // row of a tile with an 8-cell halo (two-step forward)

template <int W>
__device__ __forceinline__ float4 ld4s(const float (*s)[W], int r, int c)
{
    return *reinterpret_cast<const float4 *>(&s[r][c]);
}

__device__ __forceinline__ float4 ld4g(const float *p)
{
    return *reinterpret_cast<const float4 *>(p);
}

__device__ __forceinline__ void st4g(float *p, float4 v)
{
    *reinterpret_cast<float4 *>(p) = v;
}

// ---- TMA staging of a tile ------------------------------------------------

// A waiting thread is suspended in try_wait until the copies land or
// TMA_SUSPEND_NS pass (so it does not spin through issue slots); after
// TMA_WAIT_LIMIT rounds (about a second) it gives up.
constexpr long long TMA_WAIT_LIMIT = 1LL << 20;
constexpr unsigned TMA_SUSPEND_NS = 1000;

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// One TMA tensor copy: destination in shared memory, descriptor, and the
// start coordinates (x, z, shot, slot) of its box.  x is a multiple of 4
// floats (16 bytes), as TMA requires; z may be negative (zero fill).
struct Copy4 {
    const void *dst;
    const CUtensorMap *map;
    int x, z, s, slot;
};

// Programmatic dependent launch: wait until the launches before this one
// have completed and their writes are visible, then let the next launch in
// the stream become resident while this grid runs.  Every thread of every
// CTA waits before it touches memory that earlier launches write (so each
// launch completes after its predecessor, including CTAs that return early).
// Without the launch attribute the wait returns at once.
__device__ __forceinline__ void grid_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void issue(const Copy4 &cp, unsigned b)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(cp.dst)),
                 "l"(reinterpret_cast<unsigned long long>(cp.map)), "r"(cp.x), "r"(cp.z), "r"(cp.s), "r"(cp.slot),
                 "r"(b)
                 : "memory");
}

// Thread (0, 0) arms the CTA's mbarrier for `bytes` and issues the copies:
// the first n_early (sources no earlier launch of the stream writes) before
// the grid-dependency wait, the rest after it.  The CTA can then load what
// it needs besides the tiles while the copies are in flight.
template <int N>
__device__ __forceinline__ void stage_issue(unsigned long long *bar, const Copy4 (&cp)[N], unsigned bytes,
                                            int n_early = 0)
{
    const unsigned b = smem_addr(bar);
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    if (lead) {
#pragma unroll
        for (int i = 0; i < N; ++i)
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(cp[i].map)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (i < n_early) issue(cp[i], b);
    }
    grid_wait();
    if (lead) {
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (i >= n_early) issue(cp[i], b);
    }
}

// Every thread waits for the copies of stage_issue.  Returns false (and
// raises bit 2 of the error word) if they do not land within the wait
// limit; the whole CTA returns the same value.
__device__ __forceinline__ bool stage_wait(unsigned long long *bar, int *err)
{
    const unsigned b = smem_addr(bar);
    __syncthreads();   // the barrier is initialised before anyone waits on it
    bool ok = false;
    for (long long i = 0; i < TMA_WAIT_LIMIT && !ok; ++i) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0, %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(b), "r"(TMA_SUSPEND_NS) : "memory");
        ok = done != 0;
    }
    // bit 8: a tile copy may still be in flight into this CTA's shared memory
    // after the CTA returns, so the host retires the plan (sticky)
    if (!ok) atomicOr(err, 8);
    return __syncthreads_and(ok) != 0;   // the whole CTA takes the same branch
}

// Shot sg has no step n: every shot of the batch is active below nt_min, so
// the record length is read only near the end of the sweep.
__device__ __forceinline__ bool shot_done(const Geo &g, int sg, int n)
{
    return n >= g.nt_min && n >= g.nt[sg];
}

// T at the four cells (rr, cc..cc+3) of a staged tile of row width W.
template <int W>
__device__ __forceinline__ float4 stencil4(const float (*s)[W], int rr, int cc, float rz)
{
    float4 up[4], dn[4];
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
        up[k - 1] = ld4s(s, rr - k, cc);
        dn[k - 1] = ld4s(s, rr + k, cc);
    }
    return stencil_T(ld4s(s, rr, cc - 4), ld4s(s, rr, cc), ld4s(s, rr, cc + 4), up, dn, rz);
}

// Write f at this tile's receivers [r0, r1) (of the per-(shot, tile)
// lists) into the CSR traces of shot s, sample n.
__device__ __forceinline__ void gather(const Geo &g, int s, int r0, int r1, int n, const float *f, float *traces)
{
    if (r1 <= r0) return;
    __syncthreads();  // the tile's stores above are now visible to the block
    const long long tb = g.tr_off[s] + (long long)n * g.nrec[s];
    const int tid = threadIdx.y * BX + threadIdx.x;
    for (int i = r0 + tid; i < r1; i += BX * BY)
        traces[tb + g.trec_col[i]] = f[g.trec_pt[i]];
}

// Sponge factors of a thread's float4 column group (dgx and its negative)
// and of its RZ rows, read while the CTA's tile copies are in flight.
template <int RZ>
struct Sponge {
    float4 dgx, ndgx;
    float dz[RZ];
};

template <int RZ>
__device__ __forceinline__ Sponge<RZ> load_sponge(const Geo &g, int z0, int x)
{
    Sponge<RZ> q;
    q.dgx = x < g.pitch ? ld4g(g.dGx + x) : make_float4(0.f, 0.f, 0.f, 0.f);
    q.ndgx = neg4(q.dgx);
#pragma unroll
    for (int r = 0; r < RZ; ++r) {
        const int z = z0 + threadIdx.y + r * BY;
        q.dz[r] = z < g.NZ ? g.dGz[z] : 0.f;
    }
    return q;
}

// Forward step.  A thread owns RZ adjacent rows of its float4 column group
// and keeps the z window of each pair of them (10 rows) in registers, so
// the pair shares its z-neighbour loads (64 registers, 4 CTAs per SM).
template <int RZ>
__global__ void __launch_bounds__(BX *BY, 4) k_fwd(const Geo g, const FwdArgs a, const __grid_constant__ CUtensorMap tm_u,
                                                const __grid_constant__ CUtensorMap tm_p,
                                                const __grid_constant__ CUtensorMap tm_w)
{
    constexpr int TZ = RZ * BY, SH = TZ + 2 * HALO;
    const int s = g.s_off + blockIdx.z, sg = g.shot0 + s;   // batch-local, global shot
    if (shot_done(g, sg, a.n)) {
        grid_wait();
        return;
    }
    const int txi = blockIdx.x, tzi = blockIdx.y, tile = tzi * g.ntx + txi;
    const int z0 = tzi * TZ, x0 = txi * TX;
    extern __shared__ __align__(128) float smem[];
    __shared__ unsigned long long bar;
    Tile *su = reinterpret_cast<Tile *>(smem);                              // u^n with halo
    float(*sp)[TX] = reinterpret_cast<float(*)[TX]>(smem + SH * SW);        // u^{n-1}
    float(*swh)[TX] = reinterpret_cast<float(*)[TX]>(smem + SH * SW + TZ * TX);      // Wh
    float(*swl)[TX] = reinterpret_cast<float(*)[TX]>(smem + SH * SW + 2 * TZ * TX);  // Wl
    const long long base = (long long)s * g.field;
    // W is written only before a sweep's first launch: copied before the grid wait
    const Copy4 cp[4] = {{swh, &tm_w, x0, z0, 0, 0}, {swl, &tm_w, x0, z0, 0, 1},
                         {su, &tm_u, x0 - HALO, z0 - HALO, s, a.cur_slot}, {sp, &tm_p, x0, z0, s, a.prev_slot}};
    stage_issue(&bar, cp, (unsigned)((SH * SW + 3 * TZ * TX) * sizeof(float)), 2);
    const int xl = threadIdx.x * 4, x = x0 + xl;
    const int zb = threadIdx.y * RZ;   // this thread's RZ adjacent rows zb .. zb+RZ-1 of the tile
    Sponge<RZ> sp_;
    sp_.dgx = x < g.pitch ? ld4g(g.dGx + x) : make_float4(0.f, 0.f, 0.f, 0.f);
    sp_.ndgx = neg4(sp_.dgx);
#pragma unroll
    for (int r = 0; r < RZ; ++r) sp_.dz[r] = z0 + zb + r < g.NZ ? g.dGz[z0 + zb + r] : 0.f;
    const int src = g.src_pt[sg];
    const float wsn = g.ws[a.n];
    const int t = sg * g.ntiles + tile;
    const int r0 = g.trec_off[t], r1 = g.trec_off[t + 1];
    if (!stage_wait(&bar, g.err)) return;
    if (x < g.pitch) {
        // rows in chunks of RC; the z window of a chunk (tile rows zc-4 ..
        // zc+RC+3 of the thread's column group) sits in registers
        constexpr int RC = RZ < 2 ? RZ : 2;
#pragma unroll
        for (int c = 0; c < RZ; c += RC) {
            float4 wz[RC + 8];
#pragma unroll
            for (int k = 0; k < RC + 8; ++k) wz[k] = ld4s(su, zb + c + k, xl + HALO);
            float4 T[RC];
#pragma unroll
            for (int r = 0; r < RC; ++r) {
                float4 up[4], dn[4];
#pragma unroll
                for (int k = 1; k <= 4; ++k) {
                    up[k - 1] = wz[r + 4 - k];
                    dn[k - 1] = wz[r + 4 + k];
                }
                T[r] = stencil_T(ld4s(su, zb + c + r + HALO, xl), wz[r + 4], ld4s(su, zb + c + r + HALO, xl + 2 * HALO),
                                 up, dn, g.rz);
            }
#pragma unroll
            for (int r = 0; r < RC; ++r) {
                const int zl = zb + c + r, z = z0 + zl;
                if (z >= g.NZ) break;
                const int cell = z * g.pitch + x;
                add_source(T[r], src, (int)cell, wsn);
                if (a.t_out) __stcs(reinterpret_cast<float4 *>(a.t_out + base + cell), T[r]);
                const float4 ndG = neg_sponge4(sp_.dz[c + r], sp_.dgx, sp_.ndgx);
                const float4 uc = wz[r + 4];
                const float4 up = *reinterpret_cast<const float4 *>(&sp[zl][xl]);
                const float4 wh = *reinterpret_cast<const float4 *>(&swh[zl][xl]);
                const float4 wl = *reinterpret_cast<const float4 *>(&swl[zl][xl]);
                st4g(a.u_next + base + cell, leapfrog(ndG, uc, up, T[r], wh, wl));
                if (a.ck_cur) {
                    st4g(a.ck_cur + base + cell, uc);
                    st4g(a.ck_prev + base + cell, up);
                }
            }
        }
    }
    if (a.traces) gather(g, sg, r0, r1, a.n, a.u_next + base, a.traces);
}

// Steps n and n+1 in one launch (full-history forward sweeps).  The CTA
// stages u^n with an 8-cell halo and u^{n-1} with a 4-cell halo, advances
// its tile and the 4-cell ring around it to u^{n+1} (in shared memory, over
// u^{n-1}), then the tile to u^{n+2}.  Ring cells belong to neighbouring
// tiles, which compute them with the same operations in the same order, so
// every cell gets bitwise the value of the one-step kernel; ring cells
// outside the grid columns [0, pitch) or rows [0, NZ) are zero, as the
// one-step kernel's zero-filled halo.  T^n, T^{n+1} and u^{n+1}, u^{n+2} of
// the tile go to HBM, the traces of both steps are gathered.  A shot whose
// record ends after step n stops there.
template <int RZ>
__global__ void __launch_bounds__(BX *BY, 5) k_fwd2(const Geo g, const Fwd2Args a,
                                                 const __grid_constant__ CUtensorMap tm_u8,
                                                 const __grid_constant__ CUtensorMap tm_u4)
{
    constexpr int TZ = RZ * BY, SH = TZ + 2 * HALO, SH8 = TZ + 4 * HALO;
    constexpr int GR = SW / 4;   // float4 groups per row of tile + ring
    const int s = g.s_off + blockIdx.z, sg = g.shot0 + s;   // batch-local, global shot
    if (shot_done(g, sg, a.n)) {
        grid_wait();
        return;
    }
    const bool second = !shot_done(g, sg, a.n + 1);
    const int txi = blockIdx.x, tzi = blockIdx.y, tile = tzi * g.ntx + txi;
    const int z0 = tzi * TZ, x0 = txi * TX;
    extern __shared__ __align__(128) float smem[];
    __shared__ unsigned long long bar;
    Tile8 *sa = reinterpret_cast<Tile8 *>(smem);                // u^n, 8-cell halo
    Tile *sb = reinterpret_cast<Tile *>(smem + SH8 * SW8);      // u^{n-1}, then u^{n+1}; 4-cell halo
    const long long base = (long long)s * g.field;
    const Copy4 cp[2] = {{sa, &tm_u8, x0 - 2 * HALO, z0 - 2 * HALO, s, a.cur_slot},
                         {sb, &tm_u4, x0 - HALO, z0 - HALO, s, a.prev_slot}};
    stage_issue(&bar, cp, (unsigned)((SH8 * SW8 + SH * SW) * sizeof(float)));
    const int src = g.src_pt[sg];
    const float ws0 = g.ws[a.n], ws1 = second ? g.ws[a.n + 1] : 0.f;
    const int t = sg * g.ntiles + tile;
    const int r0 = g.trec_off[t], r1 = g.trec_off[t + 1];
    if (!stage_wait(&bar, g.err)) return;
    const int tid = threadIdx.y * BX + threadIdx.x;
    {   // step n on tile + ring; (rr, xr) in sb coordinates (origin z0 - 4, x0 - 4)
        const float wsn = ws0;
        for (int i = tid; i < SH * GR; i += BX * BY) {
            const int rr = i / GR, xr = (i - rr * GR) * 4;
            const int z = z0 - HALO + rr, x = x0 - HALO + xr;
            float4 un = make_float4(0.f, 0.f, 0.f, 0.f);
            if (z >= 0 && z < g.NZ && x >= 0 && x < g.pitch) {
                const int cell = z * g.pitch + x;
                const bool inner = rr >= HALO && rr < HALO + TZ && xr >= HALO && xr < HALO + TX;
                float4 T = stencil4(sa, rr + HALO, xr + HALO, g.rz);
                add_source(T, src, (int)cell, wsn);
                if (inner && a.t1) __stcs(reinterpret_cast<float4 *>(a.t1 + base + cell), T);
                const float4 dgx = ld4g(g.dGx + x);
                const float4 ndG = neg_sponge4(g.dGz[z], dgx, neg4(dgx));
                const float4 uc = ld4s(sa, rr + HALO, xr + HALO);
                const float4 up = ld4s(sb, rr, xr);
                const float4 wh = ld4g(a.W + cell), wl = ld4g(a.W + g.field + cell);
                un = leapfrog(ndG, uc, up, T, wh, wl);
                if (inner) st4g(a.u1 + base + cell, un);
            }
            // only this thread reads this group of u^{n-1}
            *reinterpret_cast<float4 *>(&sb[rr][xr]) = un;
        }
    }
    __syncthreads();   // u^{n+1} of tile + ring in sb, the tile's stores visible to the block
    if (a.traces) gather(g, sg, r0, r1, a.n, a.u1 + base, a.traces);
    if (!second) return;
    const int xl = threadIdx.x * 4, x = x0 + xl;
    if (x < g.pitch) {   // step n+1 on the tile
        const float4 dgx = ld4g(g.dGx + x), ndgx = neg4(dgx);
        const float wsn = ws1;
#pragma unroll
        for (int r = 0; r < RZ; ++r) {
            const int zl = threadIdx.y + r * BY, z = z0 + zl;
            if (z >= g.NZ) break;
            const int cell = z * g.pitch + x;
            float4 T = stencil4(sb, zl + HALO, xl + HALO, g.rz);
            add_source(T, src, (int)cell, wsn);
            if (a.t2) __stcs(reinterpret_cast<float4 *>(a.t2 + base + cell), T);
            const float4 ndG = neg_sponge4(g.dGz[z], dgx, ndgx);
            const float4 uc = ld4s(sb, zl + HALO, xl + HALO);
            const float4 up = ld4s(sa, zl + 2 * HALO, xl + 2 * HALO);
            const float4 wh = ld4g(a.W + cell), wl = ld4g(a.W + g.field + cell);
            st4g(a.u2 + base + cell, leapfrog(ndG, uc, up, T, wh, wl));
        }
    }
    if (a.traces) gather(g, sg, r0, r1, a.n + 1, a.u2 + base, a.traces);
}

// Born step n (eq. Born): the background u and the scattered du together.
// With 16-row tiles (BornStaged) the CTA stages everything by TMA: W (Wh, Wl) and rho before the grid-dependency wait (written only
// before a sweep), u^n and du^n with their 4-cell halos and u^{n-1}, du^{n-1}
// after it; a thread owns RZ adjacent rows of its float4 column group and
// keeps the z window of each pair of them (10 rows, for u, then for du) in
// registers.  Taller tiles would hold one or no CTA per SM that way and
// load the interior fields from global memory.  Every cell gets the operations of
// the one-field forward step, in the same order.
template <int RZ>
struct BornStaged {   // 16-row tiles: 65.5 KB of shared memory, 3 CTAs per SM
    static constexpr bool value = RZ == 2;
};

template <int RZ>
__global__ void __launch_bounds__(BX *BY, 3) k_born(const Geo g, const BornArgs a, const __grid_constant__ CUtensorMap tm_u,
                                                    const __grid_constant__ CUtensorMap tm_d,
                                                    const __grid_constant__ CUtensorMap tm_ui,
                                                    const __grid_constant__ CUtensorMap tm_di,
                                                    const __grid_constant__ CUtensorMap tm_w,
                                                    const __grid_constant__ CUtensorMap tm_r)
{
    constexpr bool STAGED = BornStaged<RZ>::value;
    constexpr int TZ = RZ * BY, SH = TZ + 2 * HALO;
    const int s = g.s_off + blockIdx.z, sg = g.shot0 + s;   // batch-local, global shot
    if (shot_done(g, sg, a.n)) {
        grid_wait();
        return;
    }
    const int txi = blockIdx.x, tzi = blockIdx.y, tile = tzi * g.ntx + txi;
    const int z0 = tzi * TZ, x0 = txi * TX;
    extern __shared__ __align__(128) float smem[];
    __shared__ unsigned long long bar;
    Tile *su = reinterpret_cast<Tile *>(smem);
    Tile *sd = su + SH;      // SH * SW * 4 bytes on: a multiple of 128
    float(*sp)[TX] = reinterpret_cast<float(*)[TX]>(smem + 2 * SH * SW);   // u^{n-1}
    float(*sdp)[TX] = sp + TZ;                                           // du^{n-1}
    float(*swh)[TX] = sdp + TZ;                                          // Wh
    float(*swl)[TX] = swh + TZ;                                          // Wl
    float(*srho)[TX] = swl + TZ;                                         // rho
    const long long base = (long long)s * g.field;
    if constexpr (STAGED) {
        const Copy4 cp[7] = {{swh, &tm_w, x0, z0, 0, 0}, {swl, &tm_w, x0, z0, 0, 1}, {srho, &tm_r, x0, z0, 0, 0},
                             {su, &tm_u, x0 - HALO, z0 - HALO, s, a.u_slot},
                             {sd, &tm_d, x0 - HALO, z0 - HALO, s, a.d_slot},
                             {sp, &tm_ui, x0, z0, s, a.u_prev_slot}, {sdp, &tm_di, x0, z0, s, a.d_prev_slot}};
        stage_issue(&bar, cp, (unsigned)((2 * SH * SW + 5 * TZ * TX) * sizeof(float)), 3);
    } else {
        const Copy4 cp[2] = {{su, &tm_u, x0 - HALO, z0 - HALO, s, a.u_slot},
                             {sd, &tm_d, x0 - HALO, z0 - HALO, s, a.d_slot}};
        stage_issue(&bar, cp, (unsigned)(2 * SH * SW * sizeof(float)));
    }
    const int xl = threadIdx.x * 4, x = x0 + xl;
    const int zb = threadIdx.y * RZ;   // this thread's RZ adjacent rows zb .. zb+RZ-1 of the tile
    Sponge<RZ> sp_;
    sp_.dgx = x < g.pitch ? ld4g(g.dGx + x) : make_float4(0.f, 0.f, 0.f, 0.f);
    sp_.ndgx = neg4(sp_.dgx);
#pragma unroll
    for (int r = 0; r < RZ; ++r) sp_.dz[r] = z0 + zb + r < g.NZ ? g.dGz[z0 + zb + r] : 0.f;
    const int src = g.src_pt[sg];
    const float wsn = g.ws[a.n];
    const int t = sg * g.ntiles + tile;
    const int r0 = g.trec_off[t], r1 = g.trec_off[t + 1];
    if (!stage_wait(&bar, g.err)) return;
    if (x < g.pitch) {
        constexpr int RC = RZ < 2 ? RZ : 2;   // rows per register window
        auto ld_tile = [&](float (*t)[TX], const float *gsrc, int zl, int cell) {
            if constexpr (STAGED) return *reinterpret_cast<const float4 *>(&t[zl][xl]);
            else return ld4g(gsrc + cell);
        };
#pragma unroll
        for (int c = 0; c < RZ; c += RC) {
            float4 wz[RC + 8];
            float4 T[RC];
            // background: the window of u^n, its stencil and source, then u^{n+1}
#pragma unroll
            for (int k = 0; k < RC + 8; ++k) wz[k] = ld4s(su, zb + c + k, xl + HALO);
#pragma unroll
            for (int r = 0; r < RC; ++r) {
                float4 up[4], dn[4];
#pragma unroll
                for (int k = 1; k <= 4; ++k) {
                    up[k - 1] = wz[r + 4 - k];
                    dn[k - 1] = wz[r + 4 + k];
                }
                T[r] = stencil_T(ld4s(su, zb + c + r + HALO, xl), wz[r + 4], ld4s(su, zb + c + r + HALO, xl + 2 * HALO),
                                 up, dn, g.rz);
                add_source(T[r], src, (int)((z0 + zb + c + r) * g.pitch + x), wsn);
            }
#pragma unroll
            for (int r = 0; r < RC; ++r) {
                const int zl = zb + c + r, z = z0 + zl;
                if (z >= g.NZ) break;
                const int cell = z * g.pitch + x;
                if (a.t_out) __stcs(reinterpret_cast<float4 *>(a.t_out + base + cell), T[r]);
                const float4 ndG = neg_sponge4(sp_.dz[c + r], sp_.dgx, sp_.ndgx);
                const float4 up = ld_tile(sp, a.u_prev + base, zl, cell);
                st4g(a.u_next + base + cell, leapfrog(ndG, wz[r + 4], up, T[r], ld_tile(swh, a.W, zl, cell),
                                                      ld_tile(swl, a.W + g.field, zl, cell)));
                if (a.ck_cur) {
                    st4g(a.ck_cur + base + cell, wz[r + 4]);
                    st4g(a.ck_prev + base + cell, up);
                }
            }
            // scattered field: the window of du^n, its stencil, the scattered
            // source W L du - W rho (L u + s) -> Wt (T_d - rho T), du^{n+1}
#pragma unroll
            for (int k = 0; k < RC + 8; ++k) wz[k] = ld4s(sd, zb + c + k, xl + HALO);
#pragma unroll
            for (int r = 0; r < RC; ++r) {
                const int zl = zb + c + r, z = z0 + zl;
                if (z >= g.NZ) break;
                const int cell = z * g.pitch + x;
                float4 up[4], dn[4];
#pragma unroll
                for (int k = 1; k <= 4; ++k) {
                    up[k - 1] = wz[r + 4 - k];
                    dn[k - 1] = wz[r + 4 + k];
                }
                const float4 Td = stencil_T(ld4s(sd, zb + c + r + HALO, xl), wz[r + 4],
                                            ld4s(sd, zb + c + r + HALO, xl + 2 * HALO), up, dn, g.rz);
                const float4 Ts = born_src(Td, ld_tile(srho, a.rho, zl, cell), T[r]);
                const float4 ndG = neg_sponge4(sp_.dz[c + r], sp_.dgx, sp_.ndgx);
                st4g(a.d_next + base + cell, leapfrog(ndG, wz[r + 4], ld_tile(sdp, a.d_prev + base, zl, cell), Ts,
                                                      ld_tile(swh, a.W, zl, cell), ld_tile(swl, a.W + g.field, zl, cell)));
            }
        }
    }
    if (a.traces) gather(g, sg, r0, r1, a.n, a.d_next + base, a.traces);
}

template <int RZ>
__global__ void __launch_bounds__(BX *BY, 4) k_adj(const Geo g, const AdjArgs a, const __grid_constant__ CUtensorMap tm_z,
                                                const __grid_constant__ CUtensorMap tm_z2,
                                                const __grid_constant__ CUtensorMap tm_t,
                                                const __grid_constant__ CUtensorMap tm_w)
{
    constexpr int TZ = RZ * BY, SH = TZ + 2 * HALO;
    const int s = g.s_off + blockIdx.z, sg = g.shot0 + s;   // batch-local, global shot
    if (shot_done(g, sg, a.n)) {
        grid_wait();
        return;
    }
    const int txi = blockIdx.x, tzi = blockIdx.y, tile = tzi * g.ntx + txi;
    const int z0 = tzi * TZ, x0 = txi * TX;
    extern __shared__ __align__(128) float smem[];
    __shared__ unsigned long long bar;
    Tile *sz = reinterpret_cast<Tile *>(smem);                                   // z^{n+1} with halo
    float(*sinj)[TX] = reinterpret_cast<float(*)[TX]>(smem + SH * SW);           // residual injection
    float(*sz2)[TX] = reinterpret_cast<float(*)[TX]>(smem + SH * SW + TZ * TX);  // z^{n+2}
    float(*st)[TX] = reinterpret_cast<float(*)[TX]>(smem + SH * SW + 2 * TZ * TX);  // T^n
    float(*swh)[TX] = reinterpret_cast<float(*)[TX]>(smem + SH * SW + 3 * TZ * TX);  // Wh
    float(*swl)[TX] = reinterpret_cast<float(*)[TX]>(smem + SH * SW + 4 * TZ * TX);  // Wl
    const long long base = (long long)s * g.field;
    // before the grid wait: W always, T^n when no launch of the sweep writes it
    const Copy4 cp[5] = {{swh, &tm_w, x0, z0, 0, 0}, {swl, &tm_w, x0, z0, 0, 1}, {st, &tm_t, x0, z0, s, a.t_slot},
                         {sz, &tm_z, x0 - HALO, z0 - HALO, s, a.z1_slot}, {sz2, &tm_z2, x0, z0, s, a.z2_slot}};
    stage_issue(&bar, cp, (unsigned)((SH * SW + 4 * TZ * TX) * sizeof(float)), a.t_early ? 3 : 2);
    // while the copies are in flight (past the grid wait): the image cells
    // this thread updates, the sponge, the residual injection
    const int xl = threadIdx.x * 4, x = x0 + xl;
    const bool xin = x < g.pitch;
    constexpr bool PRE = RZ <= 4;   // prefetch the image cells (64-row tiles: too many registers)
    float4 im[PRE ? RZ : 1];
#pragma unroll
    for (int r = 0; r < (PRE ? RZ : 0); ++r) {
        const int z = z0 + threadIdx.y + r * BY;
        if (xin && z < g.NZ) im[r] = ld4g(a.img + base + z * g.pitch + x);
    }
    const Sponge<RZ> sp_ = load_sponge<RZ>(g, z0, x);
    const int t = sg * g.ntiles + tile;
    const int r0 = g.trec_off[t], r1 = g.trec_off[t + 1];
    const bool has_rec = r1 > r0;
    const int tid = threadIdx.y * BX + threadIdx.x;
    if (has_rec) {
        for (int i = tid; i < TZ * TX / 4; i += BX * BY)
            reinterpret_cast<float4 *>(&sinj[0][0])[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        const long long tb = g.tr_off[sg] + (long long)a.n * g.nrec[sg];
        for (int i = r0 + tid; i < r1; i += BX * BY) {
            const int pt = g.trec_pt[i];
            const int zz = pt / g.pitch, xx = pt - zz * g.pitch;
            sinj[zz - z0][xx - x0] = g.inj_scale * a.resid[tb + g.trec_col[i]];
        }
    }
    if (!stage_wait(&bar, g.err)) return;   // also orders the injection tile
    if (!xin) return;
#pragma unroll
    for (int r = 0; r < RZ; ++r) {
        const int zl = threadIdx.y + r * BY, z = z0 + zl;
        if (z >= g.NZ) break;
        const int cell = z * g.pitch + x;
        const float4 Tu = *reinterpret_cast<const float4 *>(&st[zl][xl]);
        float4 Tz = stencil4(sz, zl + HALO, xl + HALO, g.rz);
        if (has_rec) {
            const float4 inj = *reinterpret_cast<const float4 *>(&sinj[zl][xl]);
            Tz = add4(Tz, inj);
        }
        const float4 ndG = neg_sponge4(sp_.dz[r], sp_.dgx, sp_.ndgx);
        const float4 z1 = ld4s(sz, zl + HALO, xl + HALO);
        const float4 z2 = *reinterpret_cast<const float4 *>(&sz2[zl][xl]);
        const float4 wh = *reinterpret_cast<const float4 *>(&swh[zl][xl]);
        const float4 wl = *reinterpret_cast<const float4 *>(&swl[zl][xl]);
        const float4 zn = leapfrog(ndG, z1, z2, Tz, wh, wl);
        // L u + s = Tu * tscale; FWI scale -1/m (= -tscale Tu 5040 dx^2 Wt/dt^2), Born -1
        float4 sc;
        if (a.born) {
            sc = make_float4(-g.tscale, -g.tscale, -g.tscale, -g.tscale);
        } else {
            sc = make_float4(__fmul_rn(g.iscale, wh.x), __fmul_rn(g.iscale, wh.y), __fmul_rn(g.iscale, wh.z),
                             __fmul_rn(g.iscale, wh.w));
        }
        const float4 imr = PRE ? im[PRE ? r : 0] : ld4g(a.img + base + cell);
        st4g(a.img + base + cell, image_acc(imr, sc, zn, Tu));
        st4g(a.z2n + base + cell, zn);
    }
}

// Wt = K/m (as the FP32 pair Wh + Wl, K = dt^2/(5040 dx^2)) and E(rho) on
// the padded grid from the physical arrays (extension E = clamp to the
// nearest physical cell); flags bad models: bit 0 non-finite or non-positive
// m, bit 1 a velocity above the plan's CFL limit (m < mcfl).
__global__ void k_prep(const Geo g, int nz, int nx, const float *m, const float *rho, float mcfl, double K,
                       float *W, float *rho_pad, int *err)
{
    const long long N = (long long)g.NZ * g.pitch;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(i / g.pitch), x = (int)(i - (long long)z * g.pitch);
        if (x >= g.NX) {          // pitch padding: the sponge table zeroes the field there
            W[i] = 0.f;
            W[g.field + i] = 0.f;
            if (rho_pad) rho_pad[i] = 0.f;
            continue;
        }
        const int jz = min(max(z - g.nb, 0), nz - 1), jx = min(max(x - g.nb, 0), nx - 1);
        const float mv = m[(long long)jz * nx + jx];
        float wh = 0.f, wl = 0.f;
        if (!(mv > 0.f) || !isfinite(mv)) {
            atomicOr(err, 1);
        } else {
            if (mv < mcfl) atomicOr(err, 2);
            const double w = K / (double)mv;
            wh = (float)w;
            wl = (float)(w - (double)wh);
        }
        W[i] = wh;
        W[g.field + i] = wl;
        if (rho_pad) rho_pad[i] = rho[(long long)jz * nx + jx];
    }
}

// grad_phys = E^T (sum over shots of the per-shot padded images), in two
// separable passes with FP64 sums in a fixed order: (1) over shots and the
// x-range of cells that physical column jx replicates, for every padded row;
// (2) over the z-range of rows that physical row jz replicates.
__global__ void k_shot_sum_x(const Geo g, int nx, const float *img, double *rowsum, int accumulate)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.NZ * nx) return;
    const int z = i / nx, jx = i - z * nx;
    const int xlo = jx == 0 ? 0 : jx + g.nb, xhi = jx == nx - 1 ? g.NX - 1 : jx + g.nb;
    double acc = accumulate ? rowsum[i] : 0.0;   // earlier batches' shots come first
    for (int s = 0; s < g.S; ++s) {
        const float *f = img + (long long)s * g.field + (long long)z * g.pitch;
        for (int x = xlo; x <= xhi; ++x) acc += (double)f[x];
    }
    rowsum[i] = acc;
}

__global__ void k_shot_sum_z(const Geo g, int nz, int nx, const double *rowsum, float *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nz * nx) return;
    const int jz = i / nx, jx = i - jz * nx;
    const int zlo = jz == 0 ? 0 : jz + g.nb, zhi = jz == nz - 1 ? g.NZ - 1 : jz + g.nb;
    double acc = 0.0;
    for (int z = zlo; z <= zhi; ++z) acc += rowsum[(long long)z * nx + jx];
    out[i] = (float)acc;
}

template <int RZ>
static size_t fwd_smem() { return ((RZ * BY + 2 * HALO) * SW + 3 * RZ * BY * TX) * sizeof(float); }
template <int RZ>
static size_t fwd2_smem() { return ((RZ * BY + 4 * HALO) * SW8 + (RZ * BY + 2 * HALO) * SW) * sizeof(float); }
template <int RZ>
static size_t born_smem()
{
    return (2 * (RZ * BY + 2 * HALO) * SW + (BornStaged<RZ>::value ? 5 * RZ * BY * TX : 0)) * sizeof(float);
}
template <int RZ>
static size_t adj_smem() { return ((RZ * BY + 2 * HALO) * SW + 5 * RZ * BY * TX) * sizeof(float); }

template <int RZ>
static cudaError_t init_tile_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(k_fwd<RZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem<RZ>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fwd2<RZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd2_smem<RZ>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_born<RZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)born_smem<RZ>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_adj<RZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adj_smem<RZ>());
    return e;
}

cudaError_t init_kernels()
{
    cudaError_t e = init_tile_kernels<2>();
    if (e == cudaSuccess) e = init_tile_kernels<4>();
    if (e == cudaSuccess) e = init_tile_kernels<8>();
    return e;
}

void launch_prep(const Geo &g, int nz, int nx, const float *m, const float *rho, float mcfl,
                 double K, float *W, float *rho_pad, int *err, cudaStream_t st)
{
    count_launch();
    k_prep<<<1216, 256, 0, st>>>(g, nz, nx, m, rho, mcfl, K, W, rho_pad, err);
}

bool encode_tile_map(CUtensorMap *m, const float *base, int NX, int NZ, int pitch, long long field, int S,
                     int slots, int tile_rows, int halo, std::string *why)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            *why = "cuTensorMapEncodeTiled not available";
            return false;
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[4] = {(cuuint64_t)NX, (cuuint64_t)NZ, (cuuint64_t)S, (cuuint64_t)slots};
    const cuuint64_t strides[3] = {(cuuint64_t)pitch * 4, (cuuint64_t)field * 4, (cuuint64_t)field * S * 4};
    const cuuint32_t box[4] = {(cuuint32_t)(TX + 2 * halo), (cuuint32_t)(tile_rows + 2 * halo), 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(base), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *why = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
        return false;
    }
    return true;
}

// Launch a step kernel, with the programmatic-serialisation attribute when pdl.
template <typename... P, typename... A>
static void launch_step(void (*k)(P...), size_t smem, const Geo &g, cudaStream_t st, bool pdl, A &&...args)
{
    count_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g.ntx, g.ntz, g.S);   // (x tiles, z tiles, shots): CTAs in tile order per shot
    cfg.blockDim = dim3(BX, BY);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);   // errors: cudaGetLastError
}

void launch_fwd(const Geo &g, const FwdArgs &a, const CUtensorMap &tm_u, const CUtensorMap &tm_p,
                const CUtensorMap &tm_w, cudaStream_t st, bool pdl)
{
    if (g.tz == 16) launch_step(k_fwd<2>, fwd_smem<2>(), g, st, pdl, g, a, tm_u, tm_p, tm_w);
    else if (g.tz == 64) launch_step(k_fwd<8>, fwd_smem<8>(), g, st, pdl, g, a, tm_u, tm_p, tm_w);
    else launch_step(k_fwd<4>, fwd_smem<4>(), g, st, pdl, g, a, tm_u, tm_p, tm_w);
}

void launch_fwd2(const Geo &g, const Fwd2Args &a, const CUtensorMap &tm_u8, const CUtensorMap &tm_u4, cudaStream_t st,
                 bool pdl)
{
    if (g.tz == 16) launch_step(k_fwd2<2>, fwd2_smem<2>(), g, st, pdl, g, a, tm_u8, tm_u4);
    else if (g.tz == 64) launch_step(k_fwd2<8>, fwd2_smem<8>(), g, st, pdl, g, a, tm_u8, tm_u4);
    else launch_step(k_fwd2<4>, fwd2_smem<4>(), g, st, pdl, g, a, tm_u8, tm_u4);
}

void launch_born(const Geo &g, const BornArgs &a, const CUtensorMap &tm_u, const CUtensorMap &tm_d,
                 const CUtensorMap &tm_ui, const CUtensorMap &tm_di, const CUtensorMap &tm_w, const CUtensorMap &tm_r,
                 cudaStream_t st, bool pdl)
{
    if (g.tz == 16) launch_step(k_born<2>, born_smem<2>(), g, st, pdl, g, a, tm_u, tm_d, tm_ui, tm_di, tm_w, tm_r);
    else if (g.tz == 64) launch_step(k_born<8>, born_smem<8>(), g, st, pdl, g, a, tm_u, tm_d, tm_ui, tm_di, tm_w, tm_r);
    else launch_step(k_born<4>, born_smem<4>(), g, st, pdl, g, a, tm_u, tm_d, tm_ui, tm_di, tm_w, tm_r);
}

void launch_adj(const Geo &g, const AdjArgs &a, const CUtensorMap &tm_z, const CUtensorMap &tm_z2,
                const CUtensorMap &tm_t, const CUtensorMap &tm_w, cudaStream_t st, bool pdl)
{
    if (g.tz == 16) launch_step(k_adj<2>, adj_smem<2>(), g, st, pdl, g, a, tm_z, tm_z2, tm_t, tm_w);
    else if (g.tz == 64) launch_step(k_adj<8>, adj_smem<8>(), g, st, pdl, g, a, tm_z, tm_z2, tm_t, tm_w);
    else launch_step(k_adj<4>, adj_smem<4>(), g, st, pdl, g, a, tm_z, tm_z2, tm_t, tm_w);
}

void launch_shot_sum(const Geo &g, int nz, int nx, const float *img, double *rowsum, bool accumulate, float *out,
                     cudaStream_t st)
{
    count_launch(out ? 2 : 1);
    const int n1 = g.NZ * nx, n2 = nz * nx;
    k_shot_sum_x<<<(n1 + 255) / 256, 256, 0, st>>>(g, nx, img, rowsum, accumulate ? 1 : 0);
    if (out) k_shot_sum_z<<<(n2 + 255) / 256, 256, 0, st>>>(g, nz, nx, rowsum, out);
}

}  // namespace aafwi
