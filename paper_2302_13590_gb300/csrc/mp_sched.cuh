// mp_sched.cuh - particle scheduling shared by the FP64 and mixed kernels.
//
// Two schedules of the paper's particle loop (Methods, "Multiprocessing";
// Results, "Thread scheduling"):
//   static  - one thread per particle on a plain grid; a warp runs as long as
//             its slowest particle (the GPU form of OpenMP `static`);
//   dynamic - a persistent grid of warps; lanes whose particle has ended are
//             refilled from an atomic queue head after every S cell-steps:
//             one ballot finds the idle lanes, one atomicAdd per warp claims
//             that many particle indices, a prefix popcount hands them out.
//             This is the GPU form of OpenMP `dynamic` (a new particle is
//             taken on completion of the current one) and keeps warps full
//             through the heavy tail of slow particles.
// Per-status counts and cell-step totals (the paper's `reduction` counters,
// Fig. 2) go to shared-memory atomics and one global atomic per block.
#pragma once

#include <math_constants.h>

#include "mp_internal.h"

namespace mp {

__device__ __forceinline__ unsigned long long fnv_step(unsigned long long h, int c)
{
    h ^= (unsigned long long)(unsigned)c;
    h *= 0x100000001b3ULL;
    return h;
}
constexpr unsigned long long FNV_INIT = 0xcbf29ce484222325ULL;

// one 32-byte timeseries record as two 16-byte streaming stores (full sector)
__device__ __forceinline__ void store_record(mp_ts_record* dst, double x, double y, double z, int cell, int st)
{
    double2 a = make_double2(x, y);
    long long zb = __double_as_longlong(z);
    int4 b = make_int4((int)(unsigned)(zb & 0xffffffffLL), (int)(zb >> 32), cell, st & 0xff);
    __stcs(reinterpret_cast<double2*>(dst), a);
    __stcs(reinterpret_cast<int4*>(dst) + 1, b);
}

// Per-status counts and cell-step totals.  A launch of one request sums them
// in shared memory and adds them once per block; a batch adds each ended
// particle's counts to its own request's counters directly.
template <class E>
__device__ __forceinline__ void flush_counters(const E& e, unsigned long long* s_cnt)
{
    __syncthreads();
    if (e.b.n_reqs != 1) return;
    unsigned long long* dst = e.b.reqs[0].o.counters;
    for (int i = threadIdx.x; i < COUNTER_ERR; i += blockDim.x)
        if (s_cnt[i]) atomicAdd(dst + i, s_cnt[i]);
}

__device__ __forceinline__ void count_ended(const Batch& b, int r, unsigned steps, int st,
                                            unsigned long long* s_cnt, bool count_status)
{
    unsigned long long* c = b.n_reqs == 1 ? s_cnt : b.reqs[r].o.counters;
    atomicAdd(c + COUNTER_STEPS, (unsigned long long)steps);
    if (count_status) atomicAdd(c + COUNTER_STATUS + (st & 7), 1ULL);
}

// A particle stopped at a non-final flow period's end: its later output
// times are written by the next period, not filled with this position.
template <class E, class S>
__device__ __forceinline__ bool paused(const E& e, const S& s)
{
    return (s.st == MP_ST_TIME || s.st == MP_ST_STEP_CAP) && !e.b.reqs[s.r].p.last;
}

// The launch's device-time window (global timer, ns), kept in the first
// request's counters: earliest block start, latest block end.
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void window_begin(const Batch& b)
{
    if (threadIdx.x == 0) atomicMax(b.reqs[0].o.counters + COUNTER_T_BEGIN, ~global_ns());
}

__device__ __forceinline__ void window_end(const Batch& b)
{
    if (threadIdx.x == 0) atomicMax(b.reqs[0].o.counters + COUNTER_T_END, global_ns());
}

// request of global particle index g (starts ascending, starts[0] = 0)
__device__ __forceinline__ int request_of(const Batch& b, long long g)
{
    int lo = 0, hi = b.n_reqs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(b.starts + mid) <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Deferred timeseries records (the GPU form of the paper's thread-exclusive
// output units, Methods, "Multiprocessing").  A lane whose step passes output
// times does not evaluate them on the spot - that would run the record
// branch for the whole warp with one or two lanes active in almost every
// step.  It pushes (pre-step position, cell, tau, slot) into its warp's
// shared-memory queue; whenever 32 requests are queued, the warp evaluates
// them together, one per lane, and writes 32 full-sector records.
// ---------------------------------------------------------------------------

constexpr int RQ_CAP = 64;   // requests per warp (>= 2 x 32)

// dynamic shared memory: one record queue per warp of the block
extern __shared__ __align__(16) unsigned char s_dyn[];

template <class E>
__device__ __forceinline__ void rq_drain(const E& e, typename E::RecQ& Q, int& qcount, bool all)
{
    const int lane = threadIdx.x & 31;
    while (qcount >= 32 || (all && qcount > 0)) {
        const int nb = qcount < 32 ? qcount : 32;
        const int base = qcount - nb;
        if (lane < nb) e.rec_eval(Q, base + lane);
        qcount = base;
        __syncwarp();
    }
}

// Queue m records per lane (output indices kn0 .. kn0+m-1 of the particle in
// this lane, evaluated from its pre-step state); warp-uniform call.
template <class E>
__device__ __forceinline__ void rq_push(const E& e, typename E::RecQ& Q, int& qcount,
                                        const typename E::State& s, long long q, int kn0, int m, int st)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int done = 0;
    while (true) {
        const int want = m - done;
        int incl = want;
        #pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += v;
        }
        const int excl = incl - want;
        const int room = RQ_CAP - qcount;
        int take = room - excl;
        take = take < 0 ? 0 : (take > want ? want : take);
        for (int r = 0; r < take; ++r) e.rec_put(Q, qcount + excl + r, s, q, kn0 + done + r, st);
        const int total = __shfl_sync(FULL, incl, 31);
        qcount += total < room ? total : room;
        done += take;
        __syncwarp();
        rq_drain(e, Q, qcount, false);
        if (!__any_sync(FULL, done < m)) break;
    }
}

// After a particle ends, its remaining output times all hold the final
// position and status.  The lanes of the warp write them together: the final
// record of each ending lane is broadcast and the 32 lanes store its slots.
template <class E>
__device__ __forceinline__ void tail_fill(const E& e, const typename E::State& s, long long q, bool ended)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    unsigned mask = __ballot_sync(FULL, ended);
    if (!mask) return;
    double x = 0.0, y = 0.0, z = 0.0;
    if (ended) e.final_pos(s, x, y, z);
    while (mask) {
        const int L = __ffs(mask) - 1;
        mask &= mask - 1;
        const double bx = __shfl_sync(FULL, x, L), by = __shfl_sync(FULL, y, L), bz = __shfl_sync(FULL, z, L);
        const int c = __shfl_sync(FULL, s.c, L), st = __shfl_sync(FULL, s.st, L), kn = __shfl_sync(FULL, s.kn, L);
        const int r = __shfl_sync(FULL, s.r, L);
        const long long qq = __shfl_sync(FULL, q, L);
        const Req& R = e.b.reqs[r];
        const int nt = R.p.n_times;
        mp_ts_record* ts = R.o.ts;
        const long long n = R.p.n;
        for (int kk = kn + lane; kk < nt; kk += 32)
            store_record(ts + (long long)kk * n + qq, bx, by, bz, c, st);
    }
}

// ---------------------------------------------------------------------------
// Pathline points (Methods, "MODPATH": pathline simulations).  Every lane
// that took a cell-step has one point to append; the warp stages them in a
// shared-memory queue and, when it is full, appends them to the requests'
// point arrays: records of one request take consecutive slots claimed by one
// atomicAdd on that request's cursor (__match_any_sync groups the lanes by
// request), so the output is dense and needs no compaction.  The order of
// points across particles is the order the warps produce them, as with the
// paper's threads appending to output units.
// ---------------------------------------------------------------------------

constexpr int PQ_CAP = 64;   // points per warp queue (>= 2 x 32)

struct PathQ {
    double x[PQ_CAP], y[PQ_CAP], z[PQ_CAP], t[PQ_CAP];
    int q[PQ_CAP], c[PQ_CAP], r[PQ_CAP];
    unsigned seq[PQ_CAP];
    unsigned char st[PQ_CAP];
};

// one 48-byte point as three 16-byte streaming stores
__device__ __forceinline__ void store_path(mp_path_record* dst, const PathQ& Q, int i)
{
    __stcs(reinterpret_cast<double2*>(dst), make_double2(Q.x[i], Q.y[i]));
    __stcs(reinterpret_cast<double2*>(dst) + 1, make_double2(Q.z[i], Q.t[i]));
    __stcs(reinterpret_cast<int4*>(dst) + 2, make_int4(Q.q[i], Q.c[i], (int)Q.seq[i], (int)Q.st[i]));
}

template <class E>
__device__ __forceinline__ void pl_flush(const E& e, PathQ& Q, int& pcount)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    __syncwarp();
    for (int base = 0; base < pcount; base += 32) {
        const int i = base + lane;
        const bool has = i < pcount;
        const int r = has ? Q.r[i] : -1;
        const unsigned peers = __match_any_sync(FULL, r);
        const int leader = __ffs(peers) - 1;
        unsigned long long pos = 0;
        if (has && lane == leader)
            pos = atomicAdd(e.b.reqs[r].o.counters + COUNTER_PATH, (unsigned long long)__popc(peers));
        pos = __shfl_sync(FULL, pos, leader) + (unsigned long long)__popc(peers & lt);
        if (has) {
            const DevOut& o = e.b.reqs[r].o;
            if ((long long)pos < o.path_cap) store_path(o.path + pos, Q, i);
        }
    }
    __syncwarp();
    pcount = 0;
}

// Stage the point of every lane with emit set (warp-uniform call).
template <class E>
__device__ __forceinline__ void pl_push(const E& e, PathQ& Q, int& pcount, const typename E::State& s, long long q,
                                        bool emit, int st)
{
    const unsigned FULL = 0xffffffffu;
    const unsigned m = __ballot_sync(FULL, emit);
    if (!m) return;
    if (pcount + __popc(m) > PQ_CAP) pl_flush(e, Q, pcount);
    if (emit) {
        const int lane = threadIdx.x & 31;
        const int slot = pcount + __popc(m & ((1u << lane) - 1u));
        double x, y, z, t;
        e.path_point(s, x, y, z, t);
        Q.x[slot] = x; Q.y[slot] = y; Q.z[slot] = z; Q.t[slot] = t;
        Q.q[slot] = (int)q; Q.c[slot] = s.c; Q.r[slot] = s.r;
        Q.seq[slot] = s.steps;
        Q.st[slot] = (unsigned char)st;
    }
    pcount += __popc(m);
    __syncwarp();
}

// A particle's first point: when its request records pathlines and this
// launch starts its line (not a later flow period); TIME (a start at or
// after the stop time) shows as the status it was released with.
template <class E, class S>
__device__ __forceinline__ bool path_start(const E& e, const S& s)
{
    const TrackParams& p = e.b.reqs[s.r].p;
    return p.pathline && !p.cont && s.st != ST_SKIP && s.c >= 0;
}

template <class E, bool TS, bool PL>
__global__ void __launch_bounds__(256, E::min_blocks(false, TS, PL)) k_track_static(E e)
{
    __shared__ unsigned long long s_cnt[N_COUNTERS];
    typename E::RecQ* s_q = reinterpret_cast<typename E::RecQ*>(s_dyn);
    for (int i = threadIdx.x; i < N_COUNTERS; i += blockDim.x) s_cnt[i] = 0ULL;
    window_begin(e.b);
    __syncthreads();
    const unsigned FULL = 0xffffffffu;
    typename E::RecQ& Q = s_q[TS ? (threadIdx.x >> 5) : 0];
    PathQ* s_p = reinterpret_cast<PathQ*>(s_dyn + (TS ? sizeof(typename E::RecQ) * (blockDim.x >> 5) : 0));
    PathQ& P = s_p[PL ? (threadIdx.x >> 5) : 0];
    int qcount = 0, pcount = 0;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long q = 0;
    typename E::State s;
    s.r = 0;
    s.steps = 0;
    s.st = ST_SKIP;
    s.c = -1;
    bool live = false, ended = false, loaded = false;
    if (g < e.b.n_total) {
        const int r = request_of(e.b, g);
        q = g - __ldg(e.b.starts + r);
        e.template load<TS>(r, q, s);
        live = s.st == MP_ST_ACTIVE;
        ended = !live && s.st != ST_SKIP;
        loaded = true;
    }
    if (PL) pl_push(e, P, pcount, s, q, loaded && path_start(e, s), s.st == MP_ST_TIME ? MP_ST_ACTIVE : s.st);
    if (TS) tail_fill(e, s, q, ended && !paused(e, s));
    if (ended) e.template finish<TS>(q, s, s_cnt);
    while (__any_sync(FULL, live)) {
        const unsigned before = s.steps;
        e.template step<TS>(q, s, live, Q, qcount);
        if (PL) pl_push(e, P, pcount, s, q, live && s.steps != before && e.b.reqs[s.r].p.pathline, s.st);
        ended = live && s.st != MP_ST_ACTIVE;
        if (TS) tail_fill(e, s, q, ended && !paused(e, s));
        if (ended) {
            e.template finish<TS>(q, s, s_cnt);
            live = false;
        }
    }
    if (TS) rq_drain(e, Q, qcount, true);
    if (PL) pl_flush(e, P, pcount);
    flush_counters(e, s_cnt);
    window_end(e.b);
}

template <class E, bool TS, bool PL>
__global__ void __launch_bounds__(256, E::min_blocks(true, TS, PL)) k_track_dynamic(E e)
{
    __shared__ unsigned long long s_cnt[N_COUNTERS];
    typename E::RecQ* s_q = reinterpret_cast<typename E::RecQ*>(s_dyn);
    for (int i = threadIdx.x; i < N_COUNTERS; i += blockDim.x) s_cnt[i] = 0ULL;
    window_begin(e.b);
    __syncthreads();
    typename E::RecQ& Q = s_q[TS ? (threadIdx.x >> 5) : 0];
    PathQ* s_p = reinterpret_cast<PathQ*>(s_dyn + (TS ? sizeof(typename E::RecQ) * (blockDim.x >> 5) : 0));
    PathQ& P = s_p[PL ? (threadIdx.x >> 5) : 0];
    int qcount = 0, pcount = 0;
    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;
    const unsigned long long n = (unsigned long long)e.b.n_total;
    const int S = e.b.steps_per_fetch > 0 ? e.b.steps_per_fetch : 1;
    long long q = -1;
    bool live = false;
    bool drained = false;
    typename E::State s;
    s.r = 0;
    s.steps = 0;
    s.st = ST_SKIP;
    s.c = -1;
    while (true) {
        const unsigned idle = __ballot_sync(FULL, !live);
        bool ended = false, loaded = false;
        if (idle && !drained) {
            const unsigned cnt = __popc(idle);
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(e.b.queue, (unsigned long long)cnt);
            base = __shfl_sync(FULL, base, 0);
            if (base + cnt >= n) drained = true;
            if (!live) {
                const unsigned long long qq = base + __popc(idle & lt_mask);
                if (qq < n) {
                    const int r = request_of(e.b, (long long)qq);
                    q = (long long)qq - __ldg(e.b.starts + r);
                    e.template load<TS>(r, q, s);
                    live = s.st == MP_ST_ACTIVE;
                    ended = !live && s.st != ST_SKIP;
                    loaded = true;
                }
            }
        }
        if (PL) pl_push(e, P, pcount, s, q, loaded && path_start(e, s), s.st == MP_ST_TIME ? MP_ST_ACTIVE : s.st);
        if (TS) tail_fill(e, s, q, ended && !paused(e, s));
        if (ended) e.template finish<TS>(q, s, s_cnt);
        if (!__any_sync(FULL, live)) {
            if (drained) break;
            continue;
        }
        for (int it = 0; it < S; ++it) {
            const unsigned before = s.steps;
            e.template step<TS>(q, s, live, Q, qcount);
            if (PL) pl_push(e, P, pcount, s, q, live && s.steps != before && e.b.reqs[s.r].p.pathline, s.st);
            ended = live && s.st != MP_ST_ACTIVE;
            if (TS) tail_fill(e, s, q, ended && !paused(e, s));
            if (ended) {
                e.template finish<TS>(q, s, s_cnt);
                live = false;
            }
        }
    }
    if (TS) rq_drain(e, Q, qcount, true);
    if (PL) pl_flush(e, P, pcount);
    flush_counters(e, s_cnt);
    window_end(e.b);
}

// One variant of the tracking kernel: opt in to more than 48 KB of dynamic
// shared memory when the queues need it, size a persistent grid by occupancy.
template <class E, bool TS, bool PL>
cudaError_t launch_variant(const E& e, int schedule, int block, int blocks_per_sm_cap, size_t smem, cudaStream_t st)
{
    auto kern = schedule == MP_SCHED_STATIC ? k_track_static<E, TS, PL> : k_track_dynamic<E, TS, PL>;
    cudaError_t err = cudaSuccess;
    if (smem > 48 * 1024) {
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    long long grid = (e.b.n_total + block - 1) / block;
    if (schedule != MP_SCHED_STATIC) {
        int dev = 0, sms = 0, per_sm = 0;
        if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
        if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
        if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem)) != cudaSuccess)
            return err;
        if (per_sm < 1) per_sm = 1;
        if (blocks_per_sm_cap > 0 && per_sm > blocks_per_sm_cap) per_sm = blocks_per_sm_cap;
        if (grid > (long long)sms * per_sm) grid = (long long)sms * per_sm;
    }
    kern<<<(unsigned)grid, block, smem, st>>>(e);
    return cudaGetLastError();
}

template <class E>
cudaError_t launch_tracking(const E& e, unsigned modes, int schedule, int block, int blocks_per_sm_cap,
                            cudaStream_t st)
{
    if (e.b.n_total <= 0) return cudaSuccess;
    if (block <= 0) block = 128;
    if (block > 256) block = 256;
    block = (block + 31) / 32 * 32;
    const bool ts = (modes & MODE_TS) != 0, pl = (modes & MODE_PATH) != 0;
    const size_t warps = (size_t)(block / 32);
    const size_t smem = (ts ? sizeof(typename E::RecQ) * warps : 0) + (pl ? sizeof(PathQ) * warps : 0);
    if (ts && pl) return launch_variant<E, true, true>(e, schedule, block, blocks_per_sm_cap, smem, st);
    if (ts) return launch_variant<E, true, false>(e, schedule, block, blocks_per_sm_cap, smem, st);
    if (pl) return launch_variant<E, false, true>(e, schedule, block, blocks_per_sm_cap, smem, st);
    return launch_variant<E, false, false>(e, schedule, block, blocks_per_sm_cap, smem, st);
}

}  // namespace mp
