// mp_noalloc.cu - tracking entry point that allocates no device memory.
//
// Some callers cannot allocate device memory at the point where they track
// particles: code that runs under a memory budget it does not control (an
// embedding application that hands out one fixed arena and forbids further
// cudaMalloc), or code that must not let a library grow the device's memory
// pool behind its back.  mp_track_noalloc serves them: the caller passes
// every input and output buffer, and the only other device memory the call
// uses is the small file-scope array below, which every GPU that loads this
// library holds until the process exits.  The call does copy its small
// host-side inputs (output times, the request descriptor) with
// cudaMemcpyAsync from pageable host memory, which may block the calling
// thread until the stream reaches the copy.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "mp_internal.h"

using namespace mp;

namespace {

// queue head, reduction counters, a copy of the output times and the same
// times as FP32 pairs, and the launch's one-entry request table
constexpr int kReqWords = (int)((sizeof(Req) + 2 * sizeof(long long) + 7) / 8);
constexpr int kScratchWords = 8 + N_COUNTERS + 2 * MP_NOALLOC_MAX_TIMES + kReqWords;
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long* g_ptr[kMaxDevices] = {};

int na_fail(int code, const std::string& m)
{
    mp::set_last_error(m.c_str());
    return code;
}

// Device address of the scratch array for the current device; taken once per
// device, by the first call on that device.
int scratch_ptr(unsigned long long** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(MP_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return na_fail(MP_ERR_INVALID_ARG, "mp_track_noalloc: device index too large");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return na_fail(MP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_ptr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_ptr[dev];
    return MP_OK;
}

int track_noalloc(const mp_field* f, const mp_noalloc_args* a, cudaStream_t s, mp_stats* stats)
{
    // the copies below read host memory that does not outlive the call, so
    // the call refuses a stream that is being captured into a graph
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &cap);
    if (ce != cudaSuccess)
        return na_fail(MP_ERR_CUDA, std::string("mp_track_noalloc: cudaStreamIsCapturing: ") + cudaGetErrorString(ce));
    if (cap != cudaStreamCaptureStatusNone)
        return na_fail(MP_ERR_INVALID_ARG, "mp_track_noalloc: the stream is capturing; call it outside stream capture");
    if (a->n < 0) return na_fail(MP_ERR_INVALID_ARG, "mp_track_noalloc: n < 0");
    const mp_track_opts* o = &a->opts;
    if ((o->mode & (MP_MODE_ENDPOINT | MP_MODE_TIMESERIES)) == 0 || (o->mode & ~3))
        return na_fail(MP_ERR_INVALID_ARG, "mp_track_noalloc: bad mode");
    if (o->precision != MP_PREC_FP64 && o->precision != MP_PREC_MIXED)
        return na_fail(MP_ERR_INVALID_ARG, "mp_track_noalloc: unknown precision");
    if (o->schedule != MP_SCHED_STATIC && o->schedule != MP_SCHED_DYNAMIC)
        return na_fail(MP_ERR_INVALID_ARG, "mp_track_noalloc: unknown schedule");
    if (std::isnan(o->t_stop)) return na_fail(MP_ERR_INVALID_ARG, "mp_track_noalloc: t_stop is NaN");
    if (!(o->weak_sink_fraction >= 0.0 && o->weak_sink_fraction <= 1.0))
        return na_fail(MP_ERR_INVALID_ARG, "mp_track_noalloc: weak_sink_fraction outside [0, 1]");
    const bool want_ts = (o->mode & MP_MODE_TIMESERIES) != 0;
    const int nt = want_ts ? o->n_times : 0;
    if (want_ts && (nt <= 0 || !o->times || !a->ts))
        return na_fail(MP_ERR_INVALID_ARG, "mp_track_noalloc: timeseries mode needs times and a record buffer");
    if (nt > MP_NOALLOC_MAX_TIMES)
        return na_fail(MP_ERR_INVALID_ARG, "mp_track_noalloc: more than MP_NOALLOC_MAX_TIMES output times (" +
                                               std::to_string(MP_NOALLOC_MAX_TIMES) + ")");
    for (int k = 0; k < nt; ++k) {
        if (!std::isfinite(o->times[k])) return na_fail(MP_ERR_NONFINITE, "mp_track_noalloc: non-finite time");
        if (k > 0 && o->times[k] < o->times[k - 1]) return na_fail(MP_ERR_INVALID_ARG, "mp_track_noalloc: times not ascending");
    }
    const mp_endpoints& ep = a->out;
    if (a->n > 0 && (!a->cell || !a->px || !a->py || !a->pz || !a->t || !a->status || !ep.cell || !ep.x || !ep.y ||
                     !ep.z || !ep.px || !ep.py || !ep.pz || !ep.t || !ep.status || !ep.steps || !ep.exit_face ||
                     !ep.hash))
        return na_fail(MP_ERR_INVALID_ARG, "mp_track_noalloc: every state and endpoint array is required");
    unsigned long long* scratch = nullptr;
    int rc = scratch_ptr(&scratch);
    if (rc != MP_OK) return rc;
    unsigned long long* queue = scratch;
    unsigned long long* counters = scratch + 8;
    double* times = reinterpret_cast<double*>(scratch + 8 + N_COUNTERS);
    float2* times_ff = reinterpret_cast<float2*>(scratch + 8 + N_COUNTERS + MP_NOALLOC_MAX_TIMES);
    // the array keeps the last call's contents: the queue head and counters
    // must start from zero
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (8 + N_COUNTERS), s);
    if (e == cudaSuccess && nt > 0)
        e = cudaMemcpyAsync(times, o->times, sizeof(double) * nt, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nt > 0) {
        float2 ff[256];
        for (int k0 = 0; k0 < nt && e == cudaSuccess; k0 += 256) {
            const int cnt = nt - k0 < 256 ? nt - k0 : 256;
            for (int k = 0; k < cnt; ++k) split_ff(o->times[k0 + k], ff[k].x, ff[k].y);
            e = cudaMemcpyAsync(times_ff + k0, ff, sizeof(float2) * cnt, cudaMemcpyHostToDevice, s);
        }
    }
    if (e != cudaSuccess) return na_fail(MP_ERR_CUDA, std::string("mp_track_noalloc: ") + cudaGetErrorString(e));
    Req* dreq = reinterpret_cast<Req*>(scratch + 8 + N_COUNTERS + 2 * MP_NOALLOC_MAX_TIMES);
    long long* dstarts = reinterpret_cast<long long*>(reinterpret_cast<char*>(dreq) + sizeof(Req));
    DevState st{a->cell, a->px, a->py, a->pz, a->t, a->status, nullptr, nullptr, nullptr};
    DevOut d{};
    d.cell = ep.cell; d.x = ep.x; d.y = ep.y; d.z = ep.z; d.px = ep.px; d.py = ep.py; d.pz = ep.pz; d.t = ep.t;
    d.status = ep.status; d.steps = ep.steps; d.exit_face = ep.exit_face;
    d.hash = reinterpret_cast<unsigned long long*>(ep.hash);
    d.ts = nt > 0 ? a->ts : nullptr;
    d.times = times;
    d.times_ff = times_ff;
    d.counters = counters;
    TrackParams p{};
    p.n = a->n;
    p.t_stop = (want_ts && !(o->mode & MP_MODE_ENDPOINT) && !(o->t_stop < INFINITY)) ? o->times[nt - 1] : o->t_stop;
    p.max_steps = o->max_steps > 0 ? o->max_steps : 1000000LL;
    p.n_times = nt;
    p.steps_per_fetch = o->steps_per_fetch > 0 ? o->steps_per_fetch : 4;
    p.update_group = (o->flags & MP_TRACK_UPDATE_GROUP) ? 1 : 0;
    p.pass_sinks = (o->flags & MP_TRACK_PASS_WEAK_SINKS) ? 1 : 0;
    p.sink_frac = o->weak_sink_fraction;
    p.cont = 0;
    p.last = 1;
    split_ff(p.t_stop, p.tstop_hi, p.tstop_lo);
    const int block = o->block > 0 ? o->block : 128;
    const DevField& fd = *mp::field_device_view(f);
    Req hreq;
    hreq.in = st;
    hreq.o = d;
    hreq.p = p;
    const long long hstarts[2] = {0, a->n};
    e = cudaMemcpyAsync(dreq, &hreq, sizeof(Req), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dstarts, hstarts, sizeof(hstarts), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return na_fail(MP_ERR_CUDA, std::string("mp_track_noalloc: ") + cudaGetErrorString(e));
    Batch b{};
    b.reqs = dreq;
    b.starts = dstarts;
    b.n_reqs = 1;
    b.n_total = a->n;
    b.steps_per_fetch = p.steps_per_fetch;
    b.queue = queue;
    e = (o->precision == MP_PREC_FP64) ? launch_track_fp64(fd, b, nt > 0 ? MODE_TS : 0u, o->schedule, block, 0, s)
                                       : launch_track_mixed(fd, b, nt > 0 ? MODE_TS : 0u, o->schedule, block, 0, s);
    if (e != cudaSuccess) return na_fail(MP_ERR_CUDA, std::string("mp_track_noalloc: launch: ") + cudaGetErrorString(e));
    if (stats) {
        unsigned long long h[N_COUNTERS];
        e = cudaMemcpyAsync(h, counters, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return na_fail(MP_ERR_CUDA, std::string("mp_track_noalloc: stats: ") + cudaGetErrorString(e));
        mp_stats out{};
        out.cell_steps = h[COUNTER_STEPS];
        for (int k = 0; k < MP_N_STATUS; ++k) out.n_status[k] = h[COUNTER_STATUS + k];
        out.t_begin_ns = h[COUNTER_T_BEGIN] ? ~h[COUNTER_T_BEGIN] : 0ULL;
        out.t_end_ns = h[COUNTER_T_END];
        out.kernel_ms = 0.0f;
        out.device_error = h[COUNTER_ERR] ? 1 : 0;
        *stats = out;
        if (h[COUNTER_ERR]) return na_fail(MP_ERR_DEVICE, "mp_track_noalloc: kernel raised its error flag");
    }
    return MP_OK;
}

}  // namespace

extern "C" int mp_track_noalloc(const mp_field* f, const mp_noalloc_args* a, void* stream, mp_stats* stats)
{
    if (!f || !a) return na_fail(MP_ERR_INVALID_ARG, "mp_track_noalloc: NULL argument");
    if (mp::field_is_usg(f)) return na_fail(MP_ERR_INVALID_ARG, "mp_track_noalloc: rectilinear grids only");
    // run on the field's device (its arrays and its copy of the scratch array
    // live there) and give the caller back the device it had current
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return na_fail(MP_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    const int dev = mp::field_device(f);
    if (dev != prev) {
        e = cudaSetDevice(dev);
        if (e != cudaSuccess) return na_fail(MP_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    }
    const int rc = track_noalloc(f, a, reinterpret_cast<cudaStream_t>(stream), stats);
    if (dev != prev) cudaSetDevice(prev);
    return rc;
}
