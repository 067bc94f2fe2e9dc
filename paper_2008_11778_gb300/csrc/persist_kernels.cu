// persist_kernels.cu -- one persistent, cooperative launch per sweep: the
// forward sweep (eq. FWD) and the adjoint sweep with the imaging condition
// (eqs. FWI_adj, adj_grad1) of every shot, all time steps, in one kernel.
//
// Decomposition: the rows of all shots (global row = shot * NZ + z) are cut
// into P contiguous strips, one per CTA (P <= number of SMs, one CTA per SM,
// co-resident by cooperative launch).  A strip's field lives in shared memory
// for the whole sweep (plus 4 halo rows above and below) and the previous
// time level in registers, so a time step touches HBM only for what the
// method must keep: the forward writes T^n = 5040 dx^2 (L u^n + s^n) of every
// cell to history slot n+1 (slot 0 stays the zero field u^0 that the per-step
// engine starts from; T^n is the quantity the imaging condition needs), the
// adjoint reads it back and accumulates the image.  Neighbouring strips
// exchange their 4 edge rows each step through a double-buffered global
// buffer and per-CTA step counters (release / acquire); every wait is bounded
// and reports AAFWI_ERR_TIMEOUT through the plan's error word instead of
// hanging.  The arithmetic per cell is stencil_math.cuh's, as in the per-step
// kernels, so results are bitwise equal to the one-launch-per-step path.
#include "internal.cuh"
#include "stencil_math.cuh"

namespace aafwi {

constexpr long long SPIN_LIMIT = 1LL << 22;   // x >= 64 ns sleep: about a second

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0 waits until both neighbours have completed `target` steps; the
// whole CTA learns the outcome.  Returns false on timeout or a raised error.
__device__ bool wait_neighbours(const PGeo &pg, int c, unsigned target, int *abort_sh)
{
    if (threadIdx.x == 0) {
        bool ok = true;
        for (int side = -1; side <= 1 && ok; side += 2) {
            const int nb = c + side;
            if (nb < 0 || nb >= pg.P) continue;
            long long it = 0;
            while (ld_acquire(pg.flags + nb) < target) {
                if (++it > SPIN_LIMIT || (*(volatile int *)pg.err & 4)) {   // own or a neighbour's timeout
                    atomicOr(pg.err, 4);
                    ok = false;
                    break;
                }
                __nanosleep(64);
            }
        }
        *abort_sh = ok ? 0 : 1;
    }
    __syncthreads();
    return *abort_sh == 0;
}

__device__ __forceinline__ void publish(const PGeo &pg, int c, unsigned steps)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        st_release(pg.flags + c, steps);
    }
}

// Copy the neighbours' edge rows (exchange buffer `par`) into the halo rows.
__device__ void load_halo(const Geo &g, const PGeo &pg, float *tile, int c, int nr, int par)
{
    const int W4 = g.pitch / 4;
    for (int i = threadIdx.x; i < 8 * W4; i += blockDim.x) {
        const int h = i / W4, x4 = i - h * W4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        int dst;
        if (h < 4) {  // rows -4..-1: bottom edge rows (slots 4..7) of CTA c-1
            if (c > 0)
                v = __ldcg(reinterpret_cast<const float4 *>(pg.exch + (((long long)par * pg.P + c - 1) * 8 + 4 + h) * g.pitch) + x4);
            dst = h;
        } else {      // rows nr..nr+3: top edge rows (slots 0..3) of CTA c+1
            if (c + 1 < pg.P)
                v = __ldcg(reinterpret_cast<const float4 *>(pg.exch + (((long long)par * pg.P + c + 1) * 8 + h - 4) * g.pitch) + x4);
            dst = nr + h;
        }
        reinterpret_cast<float4 *>(tile + (long long)dst * g.pitch)[x4] = v;
    }
}

// Publish own rows 0..3 and nr-4..nr-1 of the tile to exchange buffer `par`.
__device__ void store_edges(const Geo &g, const PGeo &pg, const float *tile, int c, int nr, int par)
{
    const int W4 = g.pitch / 4;
    for (int i = threadIdx.x; i < 8 * W4; i += blockDim.x) {
        const int h = i / W4, x4 = i - h * W4;
        const int src = h < 4 ? 4 + h : nr + h - 4;   // tile index of own row h or nr-8+h
        const float4 v = reinterpret_cast<const float4 *>(tile + (long long)src * g.pitch)[x4];
        __stcg(reinterpret_cast<float4 *>(pg.exch + (((long long)par * pg.P + c) * 8 + h) * g.pitch) + x4, v);
    }
}

// T = rz S_z + S_x for the float4 group at the centre of the register column
// w[0..8] (rows z-4..z+4 of the tile) with left / right neighbour groups L, R;
// z neighbours outside [0, NZ) of the cell's own shot read as zero.  The
// arithmetic is stencil_math.cuh's, shared with the per-step kernels.
template <bool MASK>
__device__ __forceinline__ float4 col_stencil(const Geo &g, const float4 (&w)[9], float4 L, float4 R, int z)
{
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 up[4], dn[4];
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
        up[k - 1] = !MASK || z - k >= 0 ? w[4 - k] : zero;
        dn[k - 1] = !MASK || z + k < g.NZ ? w[4 + k] : zero;
    }
    return stencil_T(L, w[4], R, up, dn, g.rz);
}

// Shared layout: two tiles of (rows_max + 8) x pitch floats, then
// rin[2][slots_max] float4 (adjoint residual injection, double-buffered by
// step parity), then SlotInfo[slots_max].  At step n tile n&1
// holds level n (own rows + the 4 halo rows above and below, refreshed from
// the neighbours) and the other tile holds level n-1 in its own rows, which
// each thread overwrites in place with level n+1 (it reads and writes only
// its own cells there).
// A step runs in two phases so that the neighbour handshake overlaps work:
//  1. the interior rows [4, nr-4), which need no halo: thread (x, y) owns
//     float4 column x of the y-th block of them and walks down it with the
//     9-row stencil column in registers;
//  2. after the neighbours' edge rows arrive, the 8 edge rows, one float4
//     group per thread at a time.
// The model is read through L1/L2.

struct Strip {
    int r0, nr, W4, ra, rb, ne;
};

// Receiver slot of a strip, resolved once per launch into shared memory so
// that the per-step gather / injection needs no chain of dependent global
// loads: lanes' receiver columns, the shot's trace base and receiver count,
// its record length, and the float4 group's index in the tile.
struct SlotInfo {
    int4 cols;
    long long tb;                 // trace offset of the shot's sample 0
    int nrec, nts, ti, pad;
};

__device__ void load_slots(const Geo &g, const PGeo &pg, const Strip &t, int s0, int s1, SlotInfo *si)
{
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    for (int q = s0 + tid; q < s1; q += nth) {
        const int grp = pg.slot_group[q];                 // global group index
        const int gr = grp / t.W4, gx = grp - gr * t.W4;
        const int s = gr / g.NZ;
        SlotInfo v;
        v.cols = pg.slot_cols[q];
        v.tb = g.tr_off[s];
        v.nrec = g.nrec[s];
        v.nts = g.nt[s];
        v.ti = (gr - t.r0 + 4) * t.W4 + gx;
        v.pad = 0;
        si[q - s0] = v;
    }
}

// inj_scale * r[n] at the four lanes of a slot (zero outside its shot's record).
__device__ __forceinline__ float4 slot_resid(const Geo &g, const float *resid, const SlotInfo &v, int n)
{
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    if (n >= 0 && n < v.nts) {
        const float *rp = resid + v.tb + (long long)n * v.nrec;
        if (v.cols.x >= 0) r.x = g.inj_scale * __ldcs(rp + v.cols.x);
        if (v.cols.y >= 0) r.y = g.inj_scale * __ldcs(rp + v.cols.y);
        if (v.cols.z >= 0) r.z = g.inj_scale * __ldcs(rp + v.cols.z);
        if (v.cols.w >= 0) r.w = g.inj_scale * __ldcs(rp + v.cols.w);
    }
    return r;
}

__device__ __forceinline__ Strip strip_of(const Geo &g, const PGeo &pg, int c)
{
    Strip t;
    t.r0 = pg.row0[c];
    t.nr = pg.row0[c + 1] - t.r0;
    t.W4 = g.pitch / 4;
    const int ni = t.nr >= 8 ? t.nr - 8 : 0;
    const int RB = (ni + blockDim.y - 1) / blockDim.y;
    t.ra = 4 + min((int)threadIdx.y * RB, ni);
    t.rb = 4 + min((int)threadIdx.y * RB + RB, ni);
    t.ne = t.nr >= 8 ? 8 : t.nr;
    return t;
}

__device__ __forceinline__ int edge_row(const Strip &t, int e) { return (t.nr < 8 || e < 4) ? e : t.nr - 8 + e; }

// Per-row model data of a float4 group: W = Wh + Wl and the sponge row factor.
struct RowW {
    float4 wh, wl;
    float dz;
};

__device__ __forceinline__ RowW load_roww(const Geo &g, const float *W, int z, int x)
{
    const long long zc = (long long)z * g.pitch + x;
    RowW q;
    q.wh = __ldg(reinterpret_cast<const float4 *>(W + zc));
    q.wl = __ldg(reinterpret_cast<const float4 *>(W + g.field + zc));
    q.dz = __ldg(g.dGz + z);
    return q;
}

// L2 prefetch of `bytes` (a multiple of 16, 16-byte aligned) starting at p.
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Forward update of float4 group (tile row r + 4, column x4) of shot s, depth z.
__device__ __forceinline__ void fwd_cell(const Geo &g, const PGeo &pg, const PFwdArgs &a, int n, const float4 *A4,
                                         float4 *B4, const float4 (&w)[9], int W4, int x4, int r, int s, int z,
                                         float wsn, float4 dgx, int nts, int srcpt, const RowW &q)
{
    const int ti = (r + 4) * W4 + x4;
    float4 out = w[4];
    if (n < nts) {
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        const int x = 4 * x4;
        const float4 L = x4 > 0 ? A4[ti - 1] : zero;
        const float4 R = x4 + 1 < W4 ? A4[ti + 1] : zero;
        float4 T = (z >= 4 && z < g.NZ - 4) ? col_stencil<false>(g, w, L, R, z) : col_stencil<true>(g, w, L, R, z);
        add_source(T, srcpt, z * g.pitch + x, wsn);
        const long long cell = (long long)s * g.field + (long long)z * g.pitch + x;
        __stcs(reinterpret_cast<float4 *>(a.hist + (long long)(n + 1) * pg.slot + cell), T);
        out = leapfrog(neg_sponge4(q.dz, dgx, neg4(dgx)), w[4], B4[ti], T, q.wh, q.wl);
    }
    B4[ti] = out;
}

// Adjoint update and imaging of float4 group (tile row r + 4, column x4).
// Image accumulation (imode): 0 none this step; 1 z^n T^n; 2 first the
// previous step's z^{n+1} T^{n+1} (z^{n+1} is the centre w[4] of the register
// column), then z^n T^n.  Pairs halve the image read-modify-write traffic
// while every cell receives the same sequence of fused multiply-adds.
__device__ __forceinline__ void adj_cell(const Geo &g, const PGeo &pg, const PAdjArgs &a, int n, const float4 *A4,
                                         float4 *B4, const float4 *rin, int s0, const float4 (&w)[9], int W4, int x4,
                                         int r, int s, int z, float4 dgx, int nts, const RowW &q, int imode,
                                         float4 Tu, float4 Tu1, int sl)
{
    const int ti = (r + 4) * W4 + x4;
    float4 out = w[4];
    if (n < nts) {
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        const int x = 4 * x4;
        const float4 L = x4 > 0 ? A4[ti - 1] : zero;
        const float4 R = x4 + 1 < W4 ? A4[ti + 1] : zero;
        float4 Tz = (z >= 4 && z < g.NZ - 4) ? col_stencil<false>(g, w, L, R, z) : col_stencil<true>(g, w, L, R, z);
        if (sl >= 0) {
            Tz = add4(Tz, rin[sl - s0]);
        }
        const long long cell = (long long)s * g.field + (long long)z * g.pitch + x;
        const float4 wh = q.wh;
        const float4 zn = leapfrog(neg_sponge4(q.dz, dgx, neg4(dgx)), w[4], B4[ti], Tz, q.wh, q.wl);
        float4 sc;
        if (a.born) {
            sc = make_float4(-g.tscale, -g.tscale, -g.tscale, -g.tscale);
        } else {
            sc = make_float4(__fmul_rn(g.iscale, wh.x), __fmul_rn(g.iscale, wh.y), __fmul_rn(g.iscale, wh.z),
                             __fmul_rn(g.iscale, wh.w));
        }
        if (imode != 0) {
            float4 *ip = reinterpret_cast<float4 *>(a.img + cell);
            float4 im = *ip;
            if (imode == 2 && n + 1 < nts) im = image_acc(im, sc, w[4], Tu1);
            im = image_acc(im, sc, zn, Tu);
            *ip = im;
        }
        out = zn;
    }
    B4[ti] = out;
}

__global__ void __launch_bounds__(PT, 1) k_fwd_persist(const Geo g, const PGeo pg, const PFwdArgs a)
{
    extern __shared__ __align__(16) float psm[];
    __shared__ int abort_sh;
    const int c = blockIdx.x;
    const Strip t = strip_of(g, pg, c);
    const int W4 = t.W4;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    const long long tsz = (long long)(pg.rows_max + 8) * g.pitch;
    float *tile[2] = {psm, psm + tsz};
    const int s0 = pg.slot_off[c], s1 = pg.slot_off[c + 1];
    SlotInfo *si = reinterpret_cast<SlotInfo *>(psm + 2 * tsz + 8LL * pg.slots_max);
    for (int i = tid; i < 2 * (pg.rows_max + 8) * W4; i += nth)
        reinterpret_cast<float4 *>(psm)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    load_slots(g, pg, t, s0, s1, si);
    const int x4 = threadIdx.x;
    const int sa = (t.r0 + t.ra) / g.NZ, za = (t.r0 + t.ra) - sa * g.NZ;
    const float4 dgx = *reinterpret_cast<const float4 *>(g.dGx + 4 * x4);
    __syncthreads();
    for (int n = 0; n < a.nt; ++n) {
        float *A = tile[n & 1];
        float *B = tile[(n + 1) & 1];
        if (c == 0 && n == a.stall_step) return;   // test hook: leave the neighbours' waits unmet
        const float4 *A4 = reinterpret_cast<const float4 *>(A);
        float4 *B4 = reinterpret_cast<float4 *>(B);
        const float wsn = g.ws[n];
        // phase 1: interior rows, no halo needed
        if (t.ra < t.rb) {
            float4 w[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) w[k] = A4[(t.ra + k) * W4 + x4];
            int s = sa, z = za;
            int nts = g.nt[s], srcpt = g.src_pt[s];
            RowW cur = load_roww(g, a.W, z, 4 * x4);
#pragma unroll
            for (int q = 0; q < RBMAX; ++q) {
                const int r = t.ra + q;
                if (r >= t.rb) break;
                // the next row's model data is loaded one row ahead
                const int zn = z + 1 == g.NZ ? 0 : z + 1;
                RowW nxt;
                if (r + 1 < t.rb) nxt = load_roww(g, a.W, zn, 4 * x4);
                fwd_cell(g, pg, a, n, A4, B4, w, W4, x4, r, s, z, wsn, dgx, nts, srcpt, cur);
#pragma unroll
                for (int k = 0; k < 8; ++k) w[k] = w[k + 1];
                if (r + 1 < t.rb) w[8] = A4[(r + 9) * W4 + x4];
                cur = nxt;
                z = zn;
                if (zn == 0 && r + 1 < t.rb) {
                    ++s;
                    nts = g.nt[s];
                    srcpt = g.src_pt[s];
                }
            }
        }
        // phase 2: neighbours' edge rows, then the strip's own edge rows
        if (n > 0) {
            if (!wait_neighbours(pg, c, (unsigned)n, &abort_sh)) return;
            load_halo(g, pg, A, c, t.nr, n & 1);
        }
        __syncthreads();
        for (int i = tid; i < t.ne * W4; i += nth) {
            const int e = i / W4, ex = i - e * W4;
            const int r = edge_row(t, e);
            const int gr = t.r0 + r, s = gr / g.NZ, z = gr - s * g.NZ;
            float4 w[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) w[k] = A4[(r + k) * W4 + ex];
            fwd_cell(g, pg, a, n, A4, B4, w, W4, ex, r, s, z, wsn, *reinterpret_cast<const float4 *>(g.dGx + 4 * ex),
                     g.nt[s], g.src_pt[s], load_roww(g, a.W, z, 4 * ex));
        }
        __syncthreads();
        store_edges(g, pg, B, c, t.nr, (n + 1) & 1);
        if (a.traces) {
            // receiver gather: sample n = u^{n+1}
            for (int j = tid; j < s1 - s0; j += nth) {
                const SlotInfo v = si[j];
                if (n >= v.nts) continue;
                const float4 u = B4[v.ti];
                float *tp = a.traces + v.tb + (long long)n * v.nrec;
                if (v.cols.x >= 0) tp[v.cols.x] = u.x;
                if (v.cols.y >= 0) tp[v.cols.y] = u.y;
                if (v.cols.z >= 0) tp[v.cols.z] = u.z;
                if (v.cols.w >= 0) tp[v.cols.w] = u.w;
            }
        }
        publish(pg, c, (unsigned)(n + 1));
    }
}

__global__ void __launch_bounds__(PT, 1) k_adj_persist(const Geo g, const PGeo pg, const PAdjArgs a)
{
    extern __shared__ __align__(16) float psm[];
    __shared__ int abort_sh;
    const int c = blockIdx.x;
    const Strip t = strip_of(g, pg, c);
    const int W4 = t.W4;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    const long long tsz = (long long)(pg.rows_max + 8) * g.pitch;
    float *tile[2] = {psm, psm + tsz};
    float4 *rin2 = reinterpret_cast<float4 *>(psm + 2 * tsz);   // [2][slots_max]
    const int s0 = pg.slot_off[c], s1 = pg.slot_off[c + 1];
    SlotInfo *si = reinterpret_cast<SlotInfo *>(psm + 2 * tsz + 8LL * pg.slots_max);
    for (int i = tid; i < 2 * (pg.rows_max + 8) * W4; i += nth)
        reinterpret_cast<float4 *>(psm)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    load_slots(g, pg, t, s0, s1, si);
    __syncthreads();
    // injection of the first step (n = nt-1); later steps are loaded one step ahead
    for (int q = tid; q < s1 - s0; q += nth) rin2[q] = slot_resid(g, a.resid, si[q], a.nt - 1);
    const int x4 = threadIdx.x;
    const int sa = (t.r0 + t.ra) / g.NZ, za = (t.r0 + t.ra) - sa * g.NZ;
    const float4 dgx = *reinterpret_cast<const float4 *>(g.dGx + 4 * x4);
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    for (int j = 0; j < a.nt; ++j) {
        const int n = a.nt - 1 - j;
        float *A = tile[j & 1];
        float *B = tile[(j + 1) & 1];
        if (c == 0 && j == a.stall_step) return;   // test hook: leave the neighbours' waits unmet
        // image pairs (n+1, n) at odd j; a last even step images alone
        const int imode = (j & 1) ? 2 : (j == a.nt - 1 ? 1 : 0);
        if (imode == 0) {   // the strip's T^n, T^{n-1} (slots n+1, n) into L2 for the next step, 16 KB per thread
            const unsigned bytes = (unsigned)t.nr * g.pitch * 4u;
            const unsigned off = (unsigned)(tid >> 1) * 16384u;
            if (off < bytes)
                prefetch_l2(reinterpret_cast<const char *>(a.hist + (long long)(n + 1 - (tid & 1)) * pg.slot +
                                                           (long long)t.r0 * g.pitch) + off,
                            min(16384u, bytes - off));
        }
        // residual injection of this step: rin[slot] = inj_scale * r[n] per lane
        // (written during the previous step); the next step's is loaded now
        // and stored after this step's cells (a thread's first slot only,
        // any further ones at the end of the step)
        const float4 *rin = rin2 + (j & 1) * pg.slots_max;
        float4 *rnext = rin2 + ((j + 1) & 1) * pg.slots_max;
        const float4 rnx = tid < s1 - s0 ? slot_resid(g, a.resid, si[tid], n - 1) : zero;
        __syncthreads();
        const float4 *A4 = reinterpret_cast<const float4 *>(A);
        float4 *B4 = reinterpret_cast<float4 *>(B);
        // phase 1: interior rows, no halo needed
        if (t.ra < t.rb) {
            float4 w[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) w[k] = A4[(t.ra + k) * W4 + x4];
            int s = sa, z = za;
            int nts = g.nt[s];
            const float *hn = a.hist + (long long)(n + 1) * pg.slot + 4 * x4;   // T^n; T^{n+1} one slot on
            const long long g0 = (long long)(t.r0 + t.ra) * g.pitch;
            RowW cur = load_roww(g, a.W, z, 4 * x4);
            float4 Tu = zero, Tu1 = zero;
            if (imode != 0) Tu = __ldcs(reinterpret_cast<const float4 *>(hn + g0));
            if (imode == 2) Tu1 = __ldcs(reinterpret_cast<const float4 *>(hn + pg.slot + g0));
            int sl = __ldg(pg.grp_slot + (long long)(t.r0 + t.ra) * W4 + x4);
#pragma unroll
            for (int q = 0; q < RBMAX; ++q) {
                const int r = t.ra + q;
                if (r >= t.rb) break;
                // the next row's model data, stored T and receiver slot are loaded one row ahead
                const int zn = z + 1 == g.NZ ? 0 : z + 1;
                RowW nxt;
                float4 Tun = zero, Tun1 = zero;
                int sln;
                if (r + 1 < t.rb) {
                    const long long go = g0 + (long long)(q + 1) * g.pitch;
                    nxt = load_roww(g, a.W, zn, 4 * x4);
                    if (imode != 0) Tun = __ldcs(reinterpret_cast<const float4 *>(hn + go));
                    if (imode == 2) Tun1 = __ldcs(reinterpret_cast<const float4 *>(hn + pg.slot + go));
                    sln = __ldg(pg.grp_slot + (long long)(t.r0 + r + 1) * W4 + x4);
                }
                adj_cell(g, pg, a, n, A4, B4, rin, s0, w, W4, x4, r, s, z, dgx, nts, cur, imode, Tu, Tu1, sl);
#pragma unroll
                for (int k = 0; k < 8; ++k) w[k] = w[k + 1];
                if (r + 1 < t.rb) w[8] = A4[(r + 9) * W4 + x4];
                cur = nxt;
                Tu = Tun;
                Tu1 = Tun1;
                sl = sln;
                z = zn;
                if (zn == 0 && r + 1 < t.rb) {
                    ++s;
                    nts = g.nt[s];
                }
            }
        }
        // phase 2: neighbours' edge rows, then the strip's own edge rows
        if (j > 0) {
            if (!wait_neighbours(pg, c, (unsigned)j, &abort_sh)) return;
            load_halo(g, pg, A, c, t.nr, j & 1);
        }
        __syncthreads();
        for (int i = tid; i < t.ne * W4; i += nth) {
            const int e = i / W4, ex = i - e * W4;
            const int r = edge_row(t, e);
            const int gr = t.r0 + r, s = gr / g.NZ, z = gr - s * g.NZ;
            float4 w[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) w[k] = A4[(r + k) * W4 + ex];
            const float *hc = a.hist + (long long)(n + 1) * pg.slot + (long long)gr * g.pitch + 4 * ex;
            const float4 Tu = imode != 0 ? __ldcs(reinterpret_cast<const float4 *>(hc)) : zero;
            const float4 Tu1 = imode == 2 ? __ldcs(reinterpret_cast<const float4 *>(hc + pg.slot)) : zero;
            adj_cell(g, pg, a, n, A4, B4, rin, s0, w, W4, ex, r, s, z, *reinterpret_cast<const float4 *>(g.dGx + 4 * ex),
                     g.nt[s], load_roww(g, a.W, z, 4 * ex), imode, Tu, Tu1, __ldg(pg.grp_slot + (long long)gr * W4 + ex));
        }
        __syncthreads();
        if (tid < s1 - s0) rnext[tid] = rnx;
        for (int q = tid + nth; q < s1 - s0; q += nth) rnext[q] = slot_resid(g, a.resid, si[q], n - 1);
        store_edges(g, pg, B, c, t.nr, (j + 1) & 1);
        publish(pg, c, (unsigned)(j + 1));
    }
}

size_t persist_smem(const Geo &g, int rows_max, int slots_max)
{
    return ((size_t)2 * (rows_max + 8) * g.pitch) * sizeof(float) +
           (size_t)slots_max * (2 * sizeof(float4) + sizeof(SlotInfo));
}

cudaError_t init_persist_kernels(size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(k_fwd_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_adj_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

cudaError_t launch_fwd_persist(const Geo &g, const PGeo &pg, const PFwdArgs &a, size_t smem, cudaStream_t st)
{
    count_launch();
    void *args[] = {(void *)&g, (void *)&pg, (void *)&a};
    return cudaLaunchCooperativeKernel((void *)k_fwd_persist, dim3(pg.P), dim3(g.pitch / 4, pg.ty), args, smem, st);
}

cudaError_t launch_adj_persist(const Geo &g, const PGeo &pg, const PAdjArgs &a, size_t smem, cudaStream_t st)
{
    count_launch();
    void *args[] = {(void *)&g, (void *)&pg, (void *)&a};
    return cudaLaunchCooperativeKernel((void *)k_adj_persist, dim3(pg.P), dim3(g.pitch / 4, pg.ty), args, smem, st);
}

}  // namespace aafwi
