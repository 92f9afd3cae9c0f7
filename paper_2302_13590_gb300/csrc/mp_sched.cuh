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
    for (int i = threadIdx.x; i < N_COUNTERS - 1; i += blockDim.x)
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

template <class E, bool TS>
__global__ void __launch_bounds__(256) k_track_static(E e)
{
    __shared__ unsigned long long s_cnt[N_COUNTERS];
    typename E::RecQ* s_q = reinterpret_cast<typename E::RecQ*>(s_dyn);
    for (int i = threadIdx.x; i < N_COUNTERS; i += blockDim.x) s_cnt[i] = 0ULL;
    __syncthreads();
    const unsigned FULL = 0xffffffffu;
    typename E::RecQ& Q = s_q[TS ? (threadIdx.x >> 5) : 0];
    int qcount = 0;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long q = 0;
    typename E::State s;
    s.r = 0;
    bool live = false, ended = false;
    if (g < e.b.n_total) {
        const int r = request_of(e.b, g);
        q = g - __ldg(e.b.starts + r);
        e.template load<TS>(r, q, s);
        live = s.st == MP_ST_ACTIVE;
        ended = !live && s.st != ST_SKIP;
    }
    if (TS) tail_fill(e, s, q, ended && !paused(e, s));
    if (ended) e.template finish<TS>(q, s, s_cnt);
    while (__any_sync(FULL, live)) {
        e.template step<TS>(q, s, live, Q, qcount);
        ended = live && s.st != MP_ST_ACTIVE;
        if (TS) tail_fill(e, s, q, ended && !paused(e, s));
        if (ended) {
            e.template finish<TS>(q, s, s_cnt);
            live = false;
        }
    }
    if (TS) rq_drain(e, Q, qcount, true);
    flush_counters(e, s_cnt);
}

template <class E, bool TS>
__global__ void __launch_bounds__(256) k_track_dynamic(E e)
{
    __shared__ unsigned long long s_cnt[N_COUNTERS];
    typename E::RecQ* s_q = reinterpret_cast<typename E::RecQ*>(s_dyn);
    for (int i = threadIdx.x; i < N_COUNTERS; i += blockDim.x) s_cnt[i] = 0ULL;
    __syncthreads();
    typename E::RecQ& Q = s_q[TS ? (threadIdx.x >> 5) : 0];
    int qcount = 0;
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
    while (true) {
        const unsigned idle = __ballot_sync(FULL, !live);
        bool ended = false;
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
                }
            }
        }
        if (TS) tail_fill(e, s, q, ended && !paused(e, s));
        if (ended) e.template finish<TS>(q, s, s_cnt);
        if (!__any_sync(FULL, live)) {
            if (drained) break;
            continue;
        }
        for (int it = 0; it < S; ++it) {
            e.template step<TS>(q, s, live, Q, qcount);
            ended = live && s.st != MP_ST_ACTIVE;
            if (TS) tail_fill(e, s, q, ended && !paused(e, s));
            if (ended) {
                e.template finish<TS>(q, s, s_cnt);
                live = false;
            }
        }
    }
    if (TS) rq_drain(e, Q, qcount, true);
    flush_counters(e, s_cnt);
}

template <class E>
cudaError_t launch_tracking(const E& e, bool ts, int schedule, int block, int blocks_per_sm_cap, cudaStream_t st)
{
    if (e.b.n_total <= 0) return cudaSuccess;
    if (block <= 0) block = 128;
    if (block > 256) block = 256;
    block = (block + 31) / 32 * 32;
    const size_t smem = ts ? sizeof(typename E::RecQ) * (size_t)(block / 32) : 0;
    if (schedule == MP_SCHED_STATIC) {
        const long long grid = (e.b.n_total + block - 1) / block;
        if (ts) k_track_static<E, true><<<(unsigned)grid, block, smem, st>>>(e);
        else k_track_static<E, false><<<(unsigned)grid, block, smem, st>>>(e);
        return cudaGetLastError();
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    if (ts) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_track_dynamic<E, true>, block, smem);
    else err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_track_dynamic<E, false>, block, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    if (blocks_per_sm_cap > 0 && per_sm > blocks_per_sm_cap) per_sm = blocks_per_sm_cap;
    long long grid = (long long)sms * per_sm;
    const long long need = (e.b.n_total + block - 1) / block;
    if (grid > need) grid = need;
    if (ts) k_track_dynamic<E, true><<<(unsigned)grid, block, smem, st>>>(e);
    else k_track_dynamic<E, false><<<(unsigned)grid, block, smem, st>>>(e);
    return cudaGetLastError();
}

}  // namespace mp
