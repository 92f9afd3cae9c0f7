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

template <class E>
__device__ __forceinline__ void flush_counters(const E& e, unsigned long long* s_cnt)
{
    __syncthreads();
    for (int i = threadIdx.x; i < N_COUNTERS - 1; i += blockDim.x)
        if (s_cnt[i]) atomicAdd(e.o.counters + i, s_cnt[i]);
}

template <class E, bool TS>
__global__ void __launch_bounds__(256) k_track_static(E e)
{
    __shared__ unsigned long long s_cnt[N_COUNTERS];
    for (int i = threadIdx.x; i < N_COUNTERS; i += blockDim.x) s_cnt[i] = 0ULL;
    __syncthreads();
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < e.p.n) {
        typename E::State s;
        e.template load<TS>(q, s);
        while (s.st == MP_ST_ACTIVE) e.template step<TS>(q, s);
        e.template finish<TS>(q, s, s_cnt);
    }
    flush_counters(e, s_cnt);
}

template <class E, bool TS>
__global__ void __launch_bounds__(256) k_track_dynamic(E e)
{
    __shared__ unsigned long long s_cnt[N_COUNTERS];
    for (int i = threadIdx.x; i < N_COUNTERS; i += blockDim.x) s_cnt[i] = 0ULL;
    __syncthreads();
    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;
    const unsigned long long n = (unsigned long long)e.p.n;
    const int S = e.p.steps_per_fetch > 0 ? e.p.steps_per_fetch : 1;
    long long q = -1;
    bool live = false;
    bool drained = false;
    typename E::State s;
    while (true) {
        const unsigned idle = __ballot_sync(FULL, !live);
        if (idle && !drained) {
            const unsigned cnt = __popc(idle);
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(e.o.queue, (unsigned long long)cnt);
            base = __shfl_sync(FULL, base, 0);
            if (base + cnt >= n) drained = true;
            if (!live) {
                const unsigned long long qq = base + __popc(idle & lt_mask);
                if (qq < n) {
                    q = (long long)qq;
                    e.template load<TS>(q, s);
                    if (s.st == MP_ST_ACTIVE) live = true;
                    else e.template finish<TS>(q, s, s_cnt);
                }
            }
        }
        if (!__any_sync(FULL, live)) {
            if (drained) break;
            continue;
        }
        for (int it = 0; it < S; ++it) {
            if (live) {
                e.template step<TS>(q, s);
                if (s.st != MP_ST_ACTIVE) {
                    e.template finish<TS>(q, s, s_cnt);
                    live = false;
                }
            }
        }
    }
    flush_counters(e, s_cnt);
}

template <class E>
cudaError_t launch_tracking(const E& e, bool ts, int schedule, int block, int blocks_per_sm_cap, cudaStream_t st)
{
    if (e.p.n <= 0) return cudaSuccess;
    if (block <= 0) block = 128;
    if (block > 256) block = 256;
    block = (block + 31) / 32 * 32;
    if (schedule == MP_SCHED_STATIC) {
        const long long grid = (e.p.n + block - 1) / block;
        if (ts) k_track_static<E, true><<<(unsigned)grid, block, 0, st>>>(e);
        else k_track_static<E, false><<<(unsigned)grid, block, 0, st>>>(e);
        return cudaGetLastError();
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    if (ts) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_track_dynamic<E, true>, block, 0);
    else err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_track_dynamic<E, false>, block, 0);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    if (blocks_per_sm_cap > 0 && per_sm > blocks_per_sm_cap) per_sm = blocks_per_sm_cap;
    long long grid = (long long)sms * per_sm;
    const long long need = (e.p.n + block - 1) / block;
    if (grid > need) grid = need;
    if (ts) k_track_dynamic<E, true><<<(unsigned)grid, block, 0, st>>>(e);
    else k_track_dynamic<E, false><<<(unsigned)grid, block, 0, st>>>(e);
    return cudaGetLastError();
}

}  // namespace mp
