// mp_api.cu - host side of the libmp C ABI (declared in include/mp.h).
//
// The library holds the flow field once on the device (the paper's central
// flow-data object reached through a pointer instead of per-thread copies;
// Methods, "Multiprocessing") and runs the particle loop as CUDA kernels.
// Request outputs come from the stream-ordered allocator so that many
// requests can be admitted, run and released without device-wide syncs.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>
#include <vector>

#include "mp_internal.h"

using namespace mp;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return MP_ERR_CUDA;
}

#define MP_CUDA(call, what)                                  \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);   \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Wait for an event with a bound; returns MP_OK, MP_ERR_TIMEOUT or MP_ERR_CUDA.
int wait_event(cudaEvent_t ev, int64_t timeout_us)
{
    if (timeout_us < 0) timeout_us = 60LL * 1000 * 1000;
    const auto t0 = std::chrono::steady_clock::now();
    int64_t sleep_us = 2;
    while (true) {
        cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return MP_OK;
        if (e != cudaErrorNotReady) return cuda_fail(e, "cudaEventQuery");
        const int64_t el = std::chrono::duration_cast<std::chrono::microseconds>(
                               std::chrono::steady_clock::now() - t0).count();
        if (el >= timeout_us) return fail(MP_ERR_TIMEOUT, "request still running after the wait limit");
        std::this_thread::sleep_for(std::chrono::microseconds(std::min<int64_t>(sleep_us, timeout_us - el)));
        sleep_us = std::min<int64_t>(sleep_us * 2, 200);
    }
}

}  // namespace

namespace {

// A group's state arrays in one buffer (256-byte aligned SoA): cell, px,
// py, pz, t, status, steps, hash, exit face.
size_t group_bytes(long long n)
{
    const size_t u = (size_t)n;
    const size_t b = align256(4 * u) + 4 * align256(8 * u) + align256(u) + align256(4 * u) + align256(8 * u) +
                     align256(u);
    return std::max<size_t>(b, 256);
}

DevState group_view(char* buf, long long n)
{
    const size_t u = (size_t)n;
    size_t off = 0;
    auto take = [&](size_t sz) { char* p = buf + off; off += align256(sz); return p; };
    DevState d{};
    d.cell = reinterpret_cast<int32_t*>(take(4 * u));
    d.px = reinterpret_cast<double*>(take(8 * u));
    d.py = reinterpret_cast<double*>(take(8 * u));
    d.pz = reinterpret_cast<double*>(take(8 * u));
    d.t = reinterpret_cast<double*>(take(8 * u));
    d.status = reinterpret_cast<uint8_t*>(take(u));
    d.steps = reinterpret_cast<uint32_t*>(take(4 * u));
    d.hash = reinterpret_cast<unsigned long long*>(take(8 * u));
    d.exit_face = reinterpret_cast<uint8_t*>(take(u));
    return d;
}

}  // namespace

struct mp_field {
    mp_ctx* ctx = nullptr;
    mp_balance balance{};  // volume balance of the face flows (at load)
    int usg = 0;           // 1: rectangular unstructured grid (u), else rectilinear (d)
    DevField d{};
    DevUsg u{};
    void* buf = nullptr;   // one allocation for all device arrays
    size_t bytes = 0;
    std::vector<double> geom;   // dims, delr, delc, dz, origin: fields with equal geom share a grid
};

struct mp_group {
    mp_ctx* ctx = nullptr;
    const mp_field* field = nullptr;
    DevState d{};
    void* buf = nullptr;   // one allocation for all state arrays
    size_t bytes = 0;
    long long n = 0;
    cudaStream_t stream = nullptr;
};

struct Request {
    mp_group* group = nullptr;
    std::vector<const mp_field*> fields;   // every field its launches read
    long long n = 0;
    int n_times = 0;
    int precision = 0;
    DevOut d{};
    void* buf = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t k0 = nullptr, k1 = nullptr;
    bool graph_owned = false;   // outputs of a captured graph: freed with it, events shared
};

struct TuneKey {
    const mp_field* f;
    int precision;
    int ts;
    bool operator<(const TuneKey& o) const
    {
        if (f != o.f) return f < o.f;
        if (precision != o.precision) return precision < o.precision;
        return ts < o.ts;
    }
};

struct mp_ctx {
    int device = 0;
    std::mutex mu;
    std::mutex host_mu;                             // one mp_track_host at a time per context
    cudaStream_t host_st[2] = {nullptr, nullptr};   // its two streams, made on first use
    std::map<TuneKey, mp_tuning> tuned;
    std::map<int64_t, Request*> reqs;
    std::set<mp_field*> fields;
    std::set<mp_group*> groups;
    std::set<mp_graph*> graphs;
    int64_t next_id = 1;
};

namespace {

// Wait (bounded) until no request of ctx still reads the given group/field.
int drain_users(mp_ctx* ctx, const mp_group* g, const mp_field* f)
{
    std::vector<cudaEvent_t> evs;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (auto& kv : ctx->reqs) {
            Request* r = kv.second;
            bool uses = g && r->group == g;
            for (const mp_field* rf : r->fields) uses = uses || (f && rf == f);
            if (uses) evs.push_back(r->k1);
        }
    }
    for (cudaEvent_t e : evs) {
        int rc = wait_event(e, -1);
        if (rc != MP_OK) return rc;
    }
    return MP_OK;
}

Request* find_req(mp_ctx* ctx, mp_req id)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->reqs.find(id);
    return it == ctx->reqs.end() ? nullptr : it->second;
}

int read_counters(Request* r, unsigned long long* h)
{
    MP_CUDA(cudaMemcpy(h, r->d.counters, sizeof(unsigned long long) * N_COUNTERS, cudaMemcpyDeviceToHost),
            "copy counters");
    return MP_OK;
}

// The balance report from per-cell (inflow, outflow) and ibound, in cell order.
mp_balance reduce_balance(const std::vector<double2>& io, const int8_t* ib, long long ncell)
{
    mp_balance b{};
    b.max_abs_cell = -1;
    for (long long c = 0; c < ncell; ++c) {
        const double in = io[(size_t)c].x, out = io[(size_t)c].y;
        if (ib[c] == 1) {
            const double r = std::fabs(in - out);
            if (b.max_abs_cell < 0 || r > b.max_abs_residual) {
                b.max_abs_residual = r;
                b.max_abs_cell = c;
            }
            if (in > 0.0) b.max_rel_residual = std::max(b.max_rel_residual, r / in);
            b.active_cells++;
        } else if (ib[c] == 2) {
            b.sink_extraction += in - out;
            b.sink_cells++;
        }
    }
    return b;
}

// per-cell (inflow, outflow) from the device, reduced on the host
int balance_from_device(const double2* dio, const int8_t* host_ib, long long ncell, mp_balance* out)
{
    std::vector<double2> io((size_t)ncell);
    if (ncell > 0)
        MP_CUDA(cudaMemcpy(io.data(), dio, sizeof(double2) * (size_t)ncell, cudaMemcpyDeviceToHost), "balance copy");
    *out = reduce_balance(io, host_ib, ncell);
    return MP_OK;
}

}  // namespace

extern "C" {

const char* mp_last_error(void) { return g_err.c_str(); }

int mp_ctx_create(int device, mp_ctx** out)
{
    if (!out) return fail(MP_ERR_INVALID_ARG, "mp_ctx_create: out is NULL");
    int ndev = 0;
    MP_CUDA(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(MP_ERR_INVALID_ARG, "mp_ctx_create: no such device");
    MP_CUDA(cudaSetDevice(device), "cudaSetDevice");
    MP_CUDA(cudaFree(nullptr), "context init");
    // keep freed request buffers in the stream-ordered pool for reuse, but
    // never by making an allocation wait for another stream's work: a
    // request freed on one stream (behind batches still queued there) would
    // otherwise hold back the next allocation on another stream, and with it
    // the overlap of independent requests
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        int no = 0;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    }
    mp_ctx* c = new mp_ctx();
    c->device = device;
    *out = c;
    return MP_OK;
}

int mp_ctx_destroy(mp_ctx* ctx)
{
    if (!ctx) return fail(MP_ERR_INVALID_ARG, "mp_ctx_destroy: NULL");
    cudaSetDevice(ctx->device);
    std::vector<mp_graph*> grs(ctx->graphs.begin(), ctx->graphs.end());
    for (mp_graph* g : grs) mp_graph_free(g);
    std::vector<mp_req> ids;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (auto& kv : ctx->reqs) ids.push_back(kv.first);
    }
    for (mp_req id : ids) mp_req_free(ctx, id);
    std::vector<mp_group*> gs(ctx->groups.begin(), ctx->groups.end());
    for (mp_group* g : gs) mp_group_free(g);
    std::vector<mp_field*> fs(ctx->fields.begin(), ctx->fields.end());
    for (mp_field* f : fs) mp_field_free(f);
    cudaDeviceSynchronize();
    for (cudaStream_t x : ctx->host_st)
        if (x) cudaStreamDestroy(x);
    delete ctx;
    return MP_OK;
}

int mp_field_load(mp_ctx* ctx, const mp_field_desc* d, mp_field** out)
{
    if (!ctx || !d || !out) return fail(MP_ERR_INVALID_ARG, "mp_field_load: NULL argument");
    if (d->nlay <= 0 || d->nrow <= 0 || d->ncol <= 0) return fail(MP_ERR_SHAPE, "mp_field_load: dims must be > 0");
    const long long nl = d->nlay, nr = d->nrow, nc = d->ncol;
    const long long ncell = nl * nr * nc;
    if (ncell > 0x7fffffffLL) return fail(MP_ERR_SHAPE, "mp_field_load: more than 2^31-1 cells");
    if (!d->delr || !d->delc || !d->dz || !d->qx || !d->qy || !d->qz || !d->porosity || !d->ibound)
        return fail(MP_ERR_INVALID_ARG, "mp_field_load: NULL array");
    for (long long a = 0; a < nc; ++a)
        if (!(d->delr[a] > 0.0) || !std::isfinite(d->delr[a])) return fail(MP_ERR_NONFINITE, "delr must be finite and > 0");
    for (long long a = 0; a < nr; ++a)
        if (!(d->delc[a] > 0.0) || !std::isfinite(d->delc[a])) return fail(MP_ERR_NONFINITE, "delc must be finite and > 0");
    for (long long a = 0; a < nl; ++a)
        if (!(d->dz[a] > 0.0) || !std::isfinite(d->dz[a])) return fail(MP_ERR_NONFINITE, "dz must be finite and > 0");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(d->origin[a])) return fail(MP_ERR_NONFINITE, "origin must be finite");
    MP_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");

    const long long nqx = nl * nr * (nc + 1), nqy = nl * (nr + 1) * nc, nqz = (nl + 1) * nr * nc;
    // persistent layout
    size_t off = 0;
    const size_t o_r64 = off; off = align256(off + sizeof(CellF64) * ncell);
    const size_t o_r32 = off; off = align256(off + sizeof(CellF32) * ncell);
    const size_t o_delr = off; off = align256(off + sizeof(double) * nc);
    const size_t o_delc = off; off = align256(off + sizeof(double) * nr);
    const size_t o_dz = off; off = align256(off + sizeof(double) * nl);
    const size_t o_xf = off; off = align256(off + sizeof(double) * (nc + 1));
    const size_t o_yf = off; off = align256(off + sizeof(double) * (nr + 1));
    const size_t o_zf = off; off = align256(off + sizeof(double) * (nl + 1));
    const size_t o_ib = off; off = align256(off + ncell);
    const size_t o_sf = off; off = align256(off + sizeof(double) * ncell);
    const size_t o_flag = off; off = align256(off + sizeof(unsigned));
    const size_t persistent = off;
    const bool dev_in = (d->flags & MP_DEVICE_PTR) != 0;
    // staging for host inputs (freed once the records are built)
    size_t soff = 0;
    const size_t o_qx = soff; soff = align256(soff + (dev_in ? 0 : sizeof(double) * nqx));
    const size_t o_qy = soff; soff = align256(soff + (dev_in ? 0 : sizeof(double) * nqy));
    const size_t o_qz = soff; soff = align256(soff + (dev_in ? 0 : sizeof(double) * nqz));
    const size_t o_por = soff; soff = align256(soff + (dev_in ? 0 : sizeof(double) * ncell));

    char* buf = nullptr;
    char* stage = nullptr;
    if (cudaMalloc(&buf, persistent) != cudaSuccess || (!dev_in && cudaMalloc(&stage, soff) != cudaSuccess)) {
        cudaGetLastError();
        if (buf) cudaFree(buf);
        return fail(MP_ERR_OOM, "mp_field_load: device allocation failed");
    }
    auto cleanup = [&](int rc) { cudaFree(buf); if (stage) cudaFree(stage); return rc; };
    std::vector<double> xf(nc + 1), yf(nr + 1), zf(nl + 1);
    xf[0] = d->origin[0];
    for (long long a = 0; a < nc; ++a) xf[a + 1] = xf[a] + d->delr[a];
    yf[0] = d->origin[1];
    for (long long a = 0; a < nr; ++a) yf[a + 1] = yf[a] + d->delc[a];
    zf[0] = d->origin[2];
    for (long long a = 0; a < nl; ++a) zf[a + 1] = zf[a] + d->dz[a];

    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaStreamCreate"));
    auto fin = [&](int rc) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
        return cleanup(rc);
    };
    const cudaMemcpyKind h2d = cudaMemcpyHostToDevice;
    const cudaMemcpyKind in_kind = dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const double* qx = dev_in ? d->qx : reinterpret_cast<double*>(stage + o_qx);
    const double* qy = dev_in ? d->qy : reinterpret_cast<double*>(stage + o_qy);
    const double* qz = dev_in ? d->qz : reinterpret_cast<double*>(stage + o_qz);
    const double* por = dev_in ? d->porosity : reinterpret_cast<double*>(stage + o_por);
    if (!dev_in) {
        if ((e = cudaMemcpyAsync(stage + o_qx, d->qx, sizeof(double) * nqx, h2d, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(stage + o_qy, d->qy, sizeof(double) * nqy, h2d, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(stage + o_qz, d->qz, sizeof(double) * nqz, h2d, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(stage + o_por, d->porosity, sizeof(double) * ncell, h2d, s)) != cudaSuccess)
            return fin(cuda_fail(e, "mp_field_load: upload"));
    }
    if ((e = cudaMemcpyAsync(buf + o_ib, d->ibound, ncell, in_kind, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(buf + o_delr, d->delr, sizeof(double) * nc, h2d, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(buf + o_delc, d->delc, sizeof(double) * nr, h2d, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(buf + o_dz, d->dz, sizeof(double) * nl, h2d, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(buf + o_xf, xf.data(), sizeof(double) * (nc + 1), h2d, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(buf + o_yf, yf.data(), sizeof(double) * (nr + 1), h2d, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(buf + o_zf, zf.data(), sizeof(double) * (nl + 1), h2d, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(buf + o_flag, 0, sizeof(unsigned), s)) != cudaSuccess)
        return fin(cuda_fail(e, "mp_field_load: upload"));
    unsigned* dflag = reinterpret_cast<unsigned*>(buf + o_flag);
    if ((e = launch_validate(qx, nqx, qy, nqy, qz, nqz, por, reinterpret_cast<int8_t*>(buf + o_ib), ncell, dflag,
                             s)) != cudaSuccess)
        return fin(cuda_fail(e, "mp_field_load: validate"));
    unsigned hflag = 0;
    if ((e = cudaMemcpyAsync(&hflag, dflag, sizeof(unsigned), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fin(cuda_fail(e, "mp_field_load: validate"));
    if (hflag & 1u) return fin(fail(MP_ERR_NONFINITE, "mp_field_load: non-finite face flow"));
    if (hflag & 2u) return fin(fail(MP_ERR_NONFINITE, "mp_field_load: porosity outside (0, 1] in an active cell"));
    if (hflag & 4u) return fin(fail(MP_ERR_INVALID_ARG, "mp_field_load: ibound outside {-1, 0, 1, 2}"));

    mp_field* f = new mp_field();
    f->ctx = ctx;
    f->d.nlay = (int)nl; f->d.nrow = (int)nr; f->d.ncol = (int)nc;
    f->d.ncell = ncell;
    f->d.rec64 = reinterpret_cast<CellF64*>(buf + o_r64);
    f->d.rec32 = reinterpret_cast<CellF32*>(buf + o_r32);
    f->d.delr = reinterpret_cast<double*>(buf + o_delr);
    f->d.delc = reinterpret_cast<double*>(buf + o_delc);
    f->d.dz = reinterpret_cast<double*>(buf + o_dz);
    f->d.xf = reinterpret_cast<double*>(buf + o_xf);
    f->d.yf = reinterpret_cast<double*>(buf + o_yf);
    f->d.zf = reinterpret_cast<double*>(buf + o_zf);
    f->d.ibound = reinterpret_cast<int8_t*>(buf + o_ib);
    f->d.sinkfrac = reinterpret_cast<double*>(buf + o_sf);
    f->d.m_ncol = div_magic((unsigned)nc);
    f->d.m_nrow = div_magic((unsigned)nr);
    double2* dio = nullptr;
    e = cudaMalloc(&dio, sizeof(double2) * (size_t)std::max(ncell, 1LL));
    if (e == cudaSuccess)
        e = launch_build_records(f->d, const_cast<CellF64*>(f->d.rec64), const_cast<CellF32*>(f->d.rec32),
                                 reinterpret_cast<double*>(buf + o_sf), dio, qx, qy, qz, por, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (stage) cudaFree(stage);
    if (e == cudaSuccess) {
        // the balance report (ibound on the host: the caller's array, or a copy)
        std::vector<int8_t> hib;
        const int8_t* ibh = d->ibound;
        if (dev_in) {
            hib.resize((size_t)ncell);
            e = cudaMemcpy(hib.data(), buf + o_ib, (size_t)ncell, cudaMemcpyDeviceToHost);
            ibh = hib.data();
        }
        if (e == cudaSuccess && balance_from_device(dio, ibh, ncell, &f->balance) != MP_OK) e = cudaErrorUnknown;
    }
    if (dio) cudaFree(dio);
    if (e != cudaSuccess) {
        delete f;
        cudaFree(buf);
        return cuda_fail(e, "mp_field_load: build records");
    }
    f->buf = buf;
    f->bytes = persistent;
    f->geom.reserve(6 + nc + nr + nl);
    f->geom.push_back((double)nl);
    f->geom.push_back((double)nr);
    f->geom.push_back((double)nc);
    f->geom.insert(f->geom.end(), d->delr, d->delr + nc);
    f->geom.insert(f->geom.end(), d->delc, d->delc + nr);
    f->geom.insert(f->geom.end(), d->dz, d->dz + nl);
    f->geom.insert(f->geom.end(), d->origin, d->origin + 3);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->fields.insert(f);
    }
    *out = f;
    return MP_OK;
}

int mp_field_free(mp_field* f)
{
    if (!f) return fail(MP_ERR_INVALID_ARG, "mp_field_free: NULL");
    mp_ctx* ctx = f->ctx;
    int rc = drain_users(ctx, nullptr, f);
    if (rc != MP_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->fields.erase(f);
    }
    cudaSetDevice(ctx->device);
    cudaFree(f->buf);
    delete f;
    return MP_OK;
}

int mp_usg_field_load(mp_ctx* ctx, const mp_usg_desc* d, mp_field** out)
{
    if (!ctx || !d || !out) return fail(MP_ERR_INVALID_ARG, "mp_usg_field_load: NULL argument");
    if (d->flags & MP_DEVICE_PTR) return fail(MP_ERR_INVALID_ARG, "mp_usg_field_load: host arrays only");
    const long long nc = d->ncell;
    if (nc <= 0 || nc > 0x7fffffffLL) return fail(MP_ERR_SHAPE, "mp_usg_field_load: ncell outside [1, 2^31)");
    if (!d->box || !d->porosity || !d->ibound || !d->face_off || !d->nbr || !d->q || !d->rect)
        return fail(MP_ERR_INVALID_ARG, "mp_usg_field_load: NULL array");
    if (d->face_off[0] != 0) return fail(MP_ERR_SHAPE, "mp_usg_field_load: face_off[0] != 0");
    for (long long k = 0; k < 6 * nc; ++k)
        if (d->face_off[k + 1] < d->face_off[k]) return fail(MP_ERR_SHAPE, "mp_usg_field_load: face_off decreases");
    const long long ns = d->face_off[6 * nc];
    if (ns > 0x7fffffffLL) return fail(MP_ERR_SHAPE, "mp_usg_field_load: more than 2^31 sub-faces");
    for (long long c = 0; c < nc; ++c) {
        for (int a = 0; a < 6; ++a)
            if (!std::isfinite(d->box[6 * c + a]) || (a >= 3 && !(d->box[6 * c + a] > 0.0)))
                return fail(MP_ERR_NONFINITE, "mp_usg_field_load: box must be finite with sizes > 0");
        const int8_t ib = d->ibound[c];
        if (ib < -1 || ib > 2) return fail(MP_ERR_INVALID_ARG, "mp_usg_field_load: ibound outside {-1, 0, 1, 2}");
        if ((ib == 1 || ib == 2) && !(d->porosity[c] > 0.0 && d->porosity[c] <= 1.0))
            return fail(MP_ERR_NONFINITE, "mp_usg_field_load: porosity outside (0, 1] in an active cell");
    }
    for (long long e = 0; e < ns; ++e) {
        if (d->nbr[e] < -1 || d->nbr[e] >= nc) return fail(MP_ERR_SHAPE, "mp_usg_field_load: neighbour out of range");
        if (!std::isfinite(d->q[e])) return fail(MP_ERR_NONFINITE, "mp_usg_field_load: non-finite flow");
        for (int a = 0; a < 4; ++a)
            if (!std::isfinite(d->rect[4 * e + a])) return fail(MP_ERR_NONFINITE, "mp_usg_field_load: non-finite rect");
    }
    MP_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    size_t off = 0;
    const size_t o_cell = off; off = align256(off + sizeof(mp::UsgCell) * (size_t)nc);
    const size_t o_geo = off; off = align256(off + sizeof(mp::UsgGeo) * (size_t)nc);
    const size_t o_fo = off; off = align256(off + sizeof(long long) * (size_t)(6 * nc + 1));
    const size_t o_sub = off; off = align256(off + sizeof(mp::UsgSub) * (size_t)std::max(ns, 1LL));
    const size_t o_ib = off; off = align256(off + (size_t)nc);
    const size_t o_sf = off; off = align256(off + sizeof(double) * (size_t)nc);
    const size_t persistent = off;
    const size_t o_box = off; off = align256(off + sizeof(double) * 6 * (size_t)nc);
    const size_t o_por = off; off = align256(off + sizeof(double) * (size_t)nc);
    char* buf = nullptr;
    if (cudaMalloc(&buf, off) != cudaSuccess) {
        cudaGetLastError();
        return fail(MP_ERR_OOM, "mp_usg_field_load: device allocation failed");
    }
    std::vector<mp::UsgSub> sub((size_t)std::max(ns, 1LL));
    for (long long e = 0; e < ns; ++e) {
        sub[e].nbr = d->nbr[e];
        sub[e].pad = 0;
        sub[e].q = d->q[e];
        for (int a = 0; a < 4; ++a) sub[e].rect[a] = d->rect[4 * e + a];
    }
    mp::DevUsg u{};
    u.ncell = nc;
    u.nsub = ns;
    u.cell = reinterpret_cast<mp::UsgCell*>(buf + o_cell);
    u.geo = reinterpret_cast<mp::UsgGeo*>(buf + o_geo);
    u.face_off = reinterpret_cast<long long*>(buf + o_fo);
    u.sub = reinterpret_cast<mp::UsgSub*>(buf + o_sub);
    u.ibound = reinterpret_cast<int8_t*>(buf + o_ib);
    u.sinkfrac = reinterpret_cast<double*>(buf + o_sf);
    cudaError_t e = cudaMemcpy(buf + o_fo, d->face_off, sizeof(long long) * (size_t)(6 * nc + 1),
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(buf + o_sub, sub.data(), sizeof(mp::UsgSub) * sub.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(buf + o_ib, d->ibound, (size_t)nc, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(buf + o_box, d->box, sizeof(double) * 6 * (size_t)nc, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(buf + o_por, d->porosity, sizeof(double) * (size_t)nc, cudaMemcpyHostToDevice);
    double2* dio = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&dio, sizeof(double2) * (size_t)std::max(nc, 1LL));
    if (e == cudaSuccess)
        e = mp::launch_build_usg(u, const_cast<mp::UsgCell*>(u.cell), const_cast<mp::UsgGeo*>(u.geo),
                                 reinterpret_cast<double*>(buf + o_sf), dio, reinterpret_cast<double*>(buf + o_box),
                                 reinterpret_cast<double*>(buf + o_por), nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    mp_balance bal{};
    if (e == cudaSuccess && balance_from_device(dio, d->ibound, nc, &bal) != MP_OK) e = cudaErrorUnknown;
    if (dio) cudaFree(dio);
    if (e != cudaSuccess) {
        cudaFree(buf);
        return cuda_fail(e, "mp_usg_field_load");
    }
    mp_field* f = new mp_field();
    f->ctx = ctx;
    f->balance = bal;
    f->usg = 1;
    f->u = u;
    f->buf = buf;
    f->bytes = persistent;
    // grid identity for flow periods: boxes and the sub-face layout
    f->geom.assign(1, -1.0);
    f->geom.insert(f->geom.end(), d->box, d->box + 6 * nc);
    for (long long k = 0; k <= 6 * nc; ++k) f->geom.push_back((double)d->face_off[k]);
    for (long long k = 0; k < ns; ++k) f->geom.push_back((double)d->nbr[k]);
    f->geom.insert(f->geom.end(), d->rect, d->rect + 4 * ns);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->fields.insert(f);
    }
    *out = f;
    return MP_OK;
}

int mp_field_balance(const mp_field* f, mp_balance* out)
{
    if (!f || !out) return fail(MP_ERR_INVALID_ARG, "mp_field_balance: NULL");
    *out = f->balance;
    return MP_OK;
}

int mp_field_bytes(const mp_field* f, size_t* bytes)
{
    if (!f || !bytes) return fail(MP_ERR_INVALID_ARG, "mp_field_bytes: NULL");
    *bytes = f->bytes;
    return MP_OK;
}

int mp_release_group(mp_ctx* ctx, const mp_field* f, const mp_release_desc* r, void* stream, mp_group** out)
{
    if (!ctx || !f || !r || !out) return fail(MP_ERR_INVALID_ARG, "mp_release_group: NULL argument");
    if (r->n < 0) return fail(MP_ERR_INVALID_ARG, "mp_release_group: n < 0");
    if (r->kind != MP_RELEASE_EXPLICIT && r->kind != MP_RELEASE_BOX)
        return fail(MP_ERR_INVALID_ARG, "mp_release_group: unknown kind");
    const long long n = r->n;
    const bool dev_in = (r->flags & MP_DEVICE_PTR) != 0;
    if (r->kind == MP_RELEASE_EXPLICIT) {
        if (n > 0 && (!r->cell || !r->local)) return fail(MP_ERR_INVALID_ARG, "mp_release_group: NULL cell/local");
        if (!dev_in) {
            for (long long q = 0; q < 3 * n; ++q)
                if (!std::isfinite(r->local[q])) return fail(MP_ERR_NONFINITE, "mp_release_group: non-finite local");
            if (r->t0)
                for (long long q = 0; q < n; ++q)
                    if (!std::isfinite(r->t0[q])) return fail(MP_ERR_NONFINITE, "mp_release_group: non-finite t0");
        }
    } else {
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(r->lo[a]) || !std::isfinite(r->hi[a]) || r->hi[a] < r->lo[a])
                return fail(MP_ERR_INVALID_ARG, "mp_release_group: box must be finite with lo <= hi");
    }
    MP_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = group_bytes(n);
    char* buf = nullptr;
    if (cudaMallocAsync(&buf, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(MP_ERR_OOM, "mp_release_group: device allocation failed");
    }
    mp_group* g = new mp_group();
    g->ctx = ctx;
    g->field = f;
    g->n = n;
    g->buf = buf;
    g->bytes = bytes;
    g->stream = s;
    g->d = group_view(buf, n);
    // a fresh particle: no steps yet (hash and exit face are read only after one)
    if (f->usg && r->kind == MP_RELEASE_BOX) {
        cudaFreeAsync(buf, s);
        delete g;
        return fail(MP_ERR_INVALID_ARG, "mp_release_group: box releases need a rectilinear grid");
    }
    cudaError_t e = cudaMemsetAsync(g->d.steps, 0, 4 * (size_t)n, s);
    if (e != cudaSuccess) {
        cudaFreeAsync(buf, s);
        delete g;
        return cuda_fail(e, "mp_release_group");
    }
    if (r->kind == MP_RELEASE_BOX) {
        e = launch_release_box(f->d, g->d, n, r->lo, r->hi, r->seed, r->id_offset, s);
    } else if (n > 0) {
        const int32_t* cell = r->cell;
        const double* local = r->local;
        const double* t0 = r->t0;
        char* tmp = nullptr;
        if (!dev_in) {
            size_t toff = 0;
            const size_t o_c = toff; toff = align256(toff + 4 * (size_t)n);
            const size_t o_l = toff; toff = align256(toff + 24 * (size_t)n);
            const size_t o_t0 = toff; toff = align256(toff + (r->t0 ? 8 * (size_t)n : 0));
            e = cudaMallocAsync(&tmp, toff, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(tmp + o_c, r->cell, 4 * (size_t)n, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(tmp + o_l, r->local, 24 * (size_t)n, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess && r->t0)
                e = cudaMemcpyAsync(tmp + o_t0, r->t0, 8 * (size_t)n, cudaMemcpyHostToDevice, s);
            cell = reinterpret_cast<int32_t*>(tmp + o_c);
            local = reinterpret_cast<double*>(tmp + o_l);
            t0 = r->t0 ? reinterpret_cast<double*>(tmp + o_t0) : nullptr;
        }
        if (e == cudaSuccess)
            e = f->usg ? launch_release_explicit_usg(f->u, g->d, n, cell, local, t0, s)
                       : launch_release_explicit(f->d, g->d, n, cell, local, t0, s);
        if (tmp) cudaFreeAsync(tmp, s);
    }
    if (e != cudaSuccess) {
        cudaFreeAsync(buf, s);
        delete g;
        return cuda_fail(e, "mp_release_group");
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->groups.insert(g);
    }
    *out = g;
    return MP_OK;
}

int mp_group_free(mp_group* g)
{
    if (!g) return fail(MP_ERR_INVALID_ARG, "mp_group_free: NULL");
    mp_ctx* ctx = g->ctx;
    int rc = drain_users(ctx, g, nullptr);
    if (rc != MP_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->groups.erase(g);
    }
    cudaSetDevice(ctx->device);
    cudaFreeAsync(g->buf, g->stream);
    delete g;
    return MP_OK;
}

int mp_group_size(const mp_group* g, int64_t* n)
{
    if (!g || !n) return fail(MP_ERR_INVALID_ARG, "mp_group_size: NULL");
    *n = g->n;
    return MP_OK;
}

}  // extern "C"

namespace {

// pathline points a request keeps (the caller's capacity, else 64 per particle)
long long path_capacity(const mp_track_opts* o, long long n)
{
    return o->path_capacity > 0 ? (long long)o->path_capacity : 64LL * n;
}

}  // namespace

extern "C" {

int mp_query_bytes(const mp_track_opts* o, int64_t n, size_t* bytes)
{
    if (!o || !bytes || n < 0) return fail(MP_ERR_INVALID_ARG, "mp_query_bytes: bad argument");
    const bool ts = (o->mode & MP_MODE_TIMESERIES) && o->n_times > 0;
    size_t b = 0;
    b += align256(4 * (size_t)n);           // cell
    b += 7 * align256(8 * (size_t)n);       // x y z px py pz t
    b += align256((size_t)n);               // status
    b += align256(4 * (size_t)n);           // steps
    b += align256((size_t)n);               // exit_face
    b += align256(8 * (size_t)n);           // hash
    b += align256(sizeof(unsigned long long) * N_COUNTERS);
    b += align256(sizeof(unsigned long long));
    if (ts) {
        b += align256(sizeof(mp_ts_record) * (size_t)o->n_times * (size_t)n);
        b += align256(sizeof(double) * (size_t)o->n_times);
        b += align256(sizeof(float2) * (size_t)o->n_times);
    }
    if (o->mode & MP_MODE_PATHLINE) b += align256(sizeof(mp_path_record) * (size_t)path_capacity(o, n));
    *bytes = b;
    return MP_OK;
}

int mp_track_launches(const mp_track_opts* o, int32_t* launches)
{
    if (!o || !launches) return fail(MP_ERR_INVALID_ARG, "mp_track_launches: NULL");
    *launches = 1;
    return MP_OK;
}

}  // extern "C"

namespace {

// Check options and allocate one request's outputs (stream-ordered); fills
// the request's device descriptor on the host side.
int prepare_request(mp_ctx* ctx, mp_group* g, const mp_track_opts* o, cudaStream_t s, Request** out,
                    mp::Req* hreq, unsigned* modes)
{
    if (!g || !o) return fail(MP_ERR_INVALID_ARG, "mp_track: NULL argument");
    if (g->ctx != ctx) return fail(MP_ERR_INVALID_ARG, "mp_track: group belongs to another context");
    if ((o->mode & (MP_MODE_ENDPOINT | MP_MODE_TIMESERIES | MP_MODE_PATHLINE)) == 0 || (o->mode & ~7))
        return fail(MP_ERR_INVALID_ARG, "mp_track: mode must be a non-empty set of MP_MODE_* bits");
    if (o->precision != MP_PREC_FP64 && o->precision != MP_PREC_MIXED && o->precision != MP_PREC_MIXED_F64T)
        return fail(MP_ERR_INVALID_ARG, "mp_track: unknown precision");
    if (g->field->usg && o->precision != MP_PREC_FP64)
        return fail(MP_ERR_INVALID_ARG, "mp_track: unstructured grids are tracked in FP64");
    if (o->schedule != MP_SCHED_STATIC && o->schedule != MP_SCHED_DYNAMIC && o->schedule != MP_SCHED_AUTO)
        return fail(MP_ERR_INVALID_ARG, "mp_track: unknown schedule");
    if (o->block < 0 || o->block > 1024) return fail(MP_ERR_INVALID_ARG, "mp_track: block outside [0, 1024]");
    if (std::isnan(o->t_stop)) return fail(MP_ERR_INVALID_ARG, "mp_track: t_stop is NaN");
    if (!(o->weak_sink_fraction >= 0.0 && o->weak_sink_fraction <= 1.0))
        return fail(MP_ERR_INVALID_ARG, "mp_track: weak_sink_fraction outside [0, 1]");
    const bool want_ts = (o->mode & MP_MODE_TIMESERIES) != 0;
    if (want_ts && (o->n_times <= 0 || !o->times))
        return fail(MP_ERR_INVALID_ARG, "mp_track: timeseries mode needs output times");
    if (o->n_times < 0) return fail(MP_ERR_INVALID_ARG, "mp_track: n_times < 0");
    const int nt = want_ts ? o->n_times : 0;
    for (int k = 0; k < nt; ++k) {
        if (!std::isfinite(o->times[k])) return fail(MP_ERR_NONFINITE, "mp_track: non-finite output time");
        if (k > 0 && o->times[k] < o->times[k - 1]) return fail(MP_ERR_INVALID_ARG, "mp_track: times not ascending");
    }
    double t_stop = o->t_stop;
    if (want_ts && !(o->mode & MP_MODE_ENDPOINT) && !(t_stop < INFINITY)) t_stop = o->times[nt - 1];
    const long long n = g->n;
    size_t bytes = 0;
    mp_track_opts oo = *o;
    oo.n_times = nt;
    mp_query_bytes(&oo, n, &bytes);
    char* buf = nullptr;
    if (cudaMallocAsync(&buf, std::max<size_t>(bytes, 256), s) != cudaSuccess) {
        cudaGetLastError();
        return fail(MP_ERR_OOM, "mp_track: device allocation failed");
    }
    Request* r = new Request();
    r->group = g;
    r->fields.push_back(g->field);
    r->n = n;
    r->n_times = nt;
    r->precision = o->precision;
    r->buf = buf;
    r->bytes = bytes;
    r->stream = s;
    size_t off = 0;
    auto take = [&](size_t sz) { char* p = buf + off; off += align256(sz); return p; };
    r->d.cell = reinterpret_cast<int32_t*>(take(4 * (size_t)n));
    r->d.x = reinterpret_cast<double*>(take(8 * (size_t)n));
    r->d.y = reinterpret_cast<double*>(take(8 * (size_t)n));
    r->d.z = reinterpret_cast<double*>(take(8 * (size_t)n));
    r->d.px = reinterpret_cast<double*>(take(8 * (size_t)n));
    r->d.py = reinterpret_cast<double*>(take(8 * (size_t)n));
    r->d.pz = reinterpret_cast<double*>(take(8 * (size_t)n));
    r->d.t = reinterpret_cast<double*>(take(8 * (size_t)n));
    r->d.status = reinterpret_cast<uint8_t*>(take((size_t)n));
    r->d.steps = reinterpret_cast<uint32_t*>(take(4 * (size_t)n));
    r->d.exit_face = reinterpret_cast<uint8_t*>(take((size_t)n));
    r->d.hash = reinterpret_cast<unsigned long long*>(take(8 * (size_t)n));
    r->d.counters = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * N_COUNTERS));
    take(sizeof(unsigned long long));   // spare word (queue head of a single-request launch)
    r->d.ts = nullptr;
    r->d.times = nullptr;
    r->d.times_ff = nullptr;
    if (nt > 0) {
        r->d.ts = reinterpret_cast<mp_ts_record*>(take(sizeof(mp_ts_record) * (size_t)nt * (size_t)n));
        r->d.times = reinterpret_cast<double*>(take(sizeof(double) * (size_t)nt));
        r->d.times_ff = reinterpret_cast<float2*>(take(sizeof(float2) * (size_t)nt));
    }
    const bool want_pl = (o->mode & MP_MODE_PATHLINE) != 0;
    r->d.path = nullptr;
    r->d.path_cap = 0;
    if (want_pl) {
        r->d.path_cap = path_capacity(o, n);
        r->d.path = reinterpret_cast<mp_path_record*>(take(sizeof(mp_path_record) * (size_t)r->d.path_cap));
    }
    cudaError_t e = cudaSuccess;
    if (nt > 0) e = cudaMemcpyAsync(const_cast<double*>(r->d.times), o->times, sizeof(double) * nt,
                                    cudaMemcpyHostToDevice, s);
    if (nt > 0 && e == cudaSuccess) {
        std::vector<float2> ff((size_t)nt);
        for (int k = 0; k < nt; ++k) split_ff(o->times[k], ff[k].x, ff[k].y);
        e = cudaMemcpyAsync(const_cast<float2*>(r->d.times_ff), ff.data(), sizeof(float2) * nt,
                            cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(r->d.counters, 0, sizeof(unsigned long long) * N_COUNTERS, s);
    if (e == cudaSuccess) e = cudaEventCreate(&r->k0);
    if (e == cudaSuccess) e = cudaEventCreate(&r->k1);
    if (e != cudaSuccess) {
        cudaFreeAsync(buf, s);
        if (r->k0) cudaEventDestroy(r->k0);
        if (r->k1) cudaEventDestroy(r->k1);
        delete r;
        return cuda_fail(e, "mp_track");
    }
    mp::TrackParams p{};
    p.n = n;
    p.t_stop = t_stop;
    p.max_steps = o->max_steps > 0 ? o->max_steps : 1000000LL;
    p.n_times = nt;
    p.steps_per_fetch = o->steps_per_fetch > 0 ? o->steps_per_fetch : 4;
    p.update_group = (o->flags & MP_TRACK_UPDATE_GROUP) ? 1 : 0;
    p.pass_sinks = (o->flags & MP_TRACK_PASS_WEAK_SINKS) ? 1 : 0;
    p.sink_frac = o->weak_sink_fraction;
    p.cont = 0;
    p.last = 1;
    split_ff(t_stop, p.tstop_hi, p.tstop_lo);
    p.pathline = want_pl ? 1 : 0;
    hreq->in = g->d;
    hreq->o = r->d;
    hreq->p = p;
    *modes = (nt > 0 ? mp::MODE_TS : 0u) | (want_pl ? mp::MODE_PATH : 0u);
    *out = r;
    return MP_OK;
}

void drop_request(Request* r)
{
    cudaFreeAsync(r->buf, r->stream);
    if (!r->graph_owned) {
        cudaEventDestroy(r->k0);
        cudaEventDestroy(r->k1);
    }
    delete r;
}

// One launch over prepared requests of one precision (Methods,
// "Multiprocessing": a single particle loop over every particle).
// ev: 1 records the requests' start events before the launch, 2 their end
// events after it (a request made of several launches records each once).
int launch_requests(const mp_field* f, Request** rs, const mp::Req* hreqs, int n, int precision, int schedule,
                    int block, int spf, unsigned modes, cudaStream_t s, unsigned ev = 3)
{
    size_t off = 0;
    const size_t o_req = off; off = align256(off + sizeof(mp::Req) * (size_t)n);
    const size_t o_st = off; off = align256(off + sizeof(long long) * ((size_t)n + 1));
    const size_t o_q = off; off = align256(off + sizeof(unsigned long long));
    char* tbl = nullptr;
    if (cudaMallocAsync(&tbl, off, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(MP_ERR_OOM, "mp_track: device allocation failed");
    }
    std::vector<long long> starts((size_t)n + 1, 0);
    for (int i = 0; i < n; ++i) starts[i + 1] = starts[i] + hreqs[i].p.n;
    cudaError_t e = cudaMemcpyAsync(tbl + o_req, hreqs, sizeof(mp::Req) * (size_t)n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tbl + o_st, starts.data(), sizeof(long long) * ((size_t)n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(tbl + o_q, 0, sizeof(unsigned long long), s);
    for (int i = 0; i < n && e == cudaSuccess && (ev & 1u); ++i) e = cudaEventRecord(rs[i]->k0, s);
    mp::Batch b{};
    b.reqs = reinterpret_cast<const mp::Req*>(tbl + o_req);
    b.starts = reinterpret_cast<const long long*>(tbl + o_st);
    b.n_reqs = n;
    b.n_total = starts[n];
    b.steps_per_fetch = spf > 0 ? spf : 4;
    b.queue = reinterpret_cast<unsigned long long*>(tbl + o_q);
    const int blk = block > 0 ? block : 128;
    if (e == cudaSuccess) {
        const mp::DevField& fd = *mp::field_device_view(f);
        if (f->usg) e = launch_track_usg(f->u, b, modes, schedule, blk, 0, s);
        else e = (precision == MP_PREC_FP64)    ? launch_track_fp64(fd, b, modes, schedule, blk, 0, s)
                 : (precision == MP_PREC_MIXED) ? launch_track_mixed(fd, b, modes, schedule, blk, 0, s)
                                                : launch_track_mixed_f64t(fd, b, modes, schedule, blk, 0, s);
        if (e == cudaSuccess) e = mp::launch_spread_window(b, s);
    }
    for (int i = 0; i < n && e == cudaSuccess && (ev & 2u); ++i) e = cudaEventRecord(rs[i]->k1, s);
    cudaFreeAsync(tbl, s);
    if (e != cudaSuccess) return cuda_fail(e, "mp_track: launch");
    return MP_OK;
}

// Launch configuration of a request: as given, or for MP_SCHED_AUTO the
// tuned one for (field, precision, timeseries) if there is one.
void resolve_launch(mp_ctx* ctx, const mp_field* f, int precision, bool ts, const mp_track_opts& o, int* sched,
                    int* blk, int* spf)
{
    *sched = o.schedule;
    *blk = o.block;
    *spf = o.steps_per_fetch;
    if (*sched != MP_SCHED_AUTO) return;
    *sched = MP_SCHED_DYNAMIC;
    *blk = 128;
    *spf = 4;
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->tuned.find(TuneKey{f, precision, ts ? 1 : 0});
    if (it != ctx->tuned.end()) {
        *sched = it->second.schedule;
        *blk = it->second.block;
        *spf = it->second.steps_per_fetch;
    }
}

// The same state arrays at another base address (a copy of the group's buffer).
DevState rebase(const DevState& d, const void* from, void* to)
{
    auto mv = [&](auto* ptr) {
        using T = std::remove_pointer_t<decltype(ptr)>;
        return reinterpret_cast<T*>(static_cast<char*>(to) +
                                    (reinterpret_cast<const char*>(ptr) - static_cast<const char*>(from)));
    };
    DevState r{};
    r.cell = mv(d.cell);
    r.px = mv(d.px);
    r.py = mv(d.py);
    r.pz = mv(d.pz);
    r.t = mv(d.t);
    r.status = mv(d.status);
    r.steps = mv(d.steps);
    r.hash = mv(d.hash);
    r.exit_face = mv(d.exit_face);
    return r;
}

mp_req register_request(mp_ctx* ctx, Request* r)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    const int64_t id = ctx->next_id++;
    ctx->reqs[id] = r;
    return id;
}

}  // namespace

extern "C" {

int mp_track(mp_ctx* ctx, mp_group* g, const mp_track_opts* o, void* stream, mp_req* out)
{
    if (!ctx || !g || !o || !out) return fail(MP_ERR_INVALID_ARG, "mp_track: NULL argument");
    return mp_track_batch(ctx, 1, &g, o, stream, out);
}

int mp_track_batch(mp_ctx* ctx, int n, mp_group* const* groups, const mp_track_opts* opts, void* stream,
                   mp_req* out)
{
    if (!ctx || !groups || !opts || !out || n < 0) return fail(MP_ERR_INVALID_ARG, "mp_track_batch: bad argument");
    if (n >= (1 << 24)) return fail(MP_ERR_INVALID_ARG, "mp_track_batch: more than 2^24 - 1 requests");
    if (n == 0) return MP_OK;
    for (int i = 0; i < n; ++i) {
        if (!groups[i]) return fail(MP_ERR_INVALID_ARG, "mp_track_batch: NULL group");
        if (groups[i]->field != groups[0]->field)
            return fail(MP_ERR_INVALID_ARG, "mp_track_batch: all groups must be released on the same field");
    }
    MP_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<Request*> rs((size_t)n, nullptr);
    std::vector<mp::Req> hr((size_t)n);
    std::vector<char> ts((size_t)n, 0);
    for (int i = 0; i < n; ++i) {
        unsigned md = 0;
        const int rc = prepare_request(ctx, groups[i], &opts[i], s, &rs[i], &hr[i], &md);
        if (rc != MP_OK) {
            for (int k = 0; k < i; ++k) drop_request(rs[k]);
            return rc;
        }
        ts[i] = (char)md;
    }
    // one launch per precision; launch options of the first request of each
    for (int prec = 0; prec < 3; ++prec) {
        std::vector<Request*> sel;
        std::vector<mp::Req> sreq;
        unsigned any_modes = 0;
        int first = -1;
        for (int i = 0; i < n; ++i)
            if (opts[i].precision == prec) {
                if (first < 0) first = i;
                sel.push_back(rs[i]);
                sreq.push_back(hr[i]);
                any_modes |= (unsigned)ts[i];
            }
        if (sel.empty()) continue;
        int sched = 0, blk = 0, spf = 0;
        resolve_launch(ctx, groups[0]->field, prec, (any_modes & mp::MODE_TS) != 0, opts[first], &sched, &blk, &spf);
        const int rc = launch_requests(groups[0]->field, sel.data(), sreq.data(), (int)sel.size(), prec,
                                       sched, blk, spf, any_modes, s);
        if (rc != MP_OK) {
            cudaStreamSynchronize(s);
            for (int k = 0; k < n; ++k) drop_request(rs[k]);
            return rc;
        }
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (int i = 0; i < n; ++i) {
            const int64_t id = ctx->next_id++;
            ctx->reqs[id] = rs[i];
            out[i] = id;
        }
    }
    return MP_OK;
}

int mp_group_set_field(mp_group* g, const mp_field* f)
{
    if (!g || !f) return fail(MP_ERR_INVALID_ARG, "mp_group_set_field: NULL argument");
    if (f->ctx != g->ctx) return fail(MP_ERR_INVALID_ARG, "mp_group_set_field: field belongs to another context");
    if (f->geom != g->field->geom)
        return fail(MP_ERR_SHAPE, "mp_group_set_field: the field's grid differs from the group's");
    g->field = f;
    return MP_OK;
}

int mp_track_periods(mp_ctx* ctx, mp_group* g, int n_periods, const mp_field* const* fields, const double* t_end,
                     const mp_track_opts* o, void* stream, mp_req* out)
{
    if (!ctx || !g || !o || !out || !fields || n_periods < 1)
        return fail(MP_ERR_INVALID_ARG, "mp_track_periods: bad argument");
    if (n_periods > 1 && !t_end) return fail(MP_ERR_INVALID_ARG, "mp_track_periods: NULL t_end");
    for (int p = 0; p < n_periods; ++p) {
        if (!fields[p]) return fail(MP_ERR_INVALID_ARG, "mp_track_periods: NULL field");
        if (fields[p]->ctx != ctx) return fail(MP_ERR_INVALID_ARG, "mp_track_periods: field of another context");
        if (fields[p]->geom != g->field->geom)
            return fail(MP_ERR_SHAPE, "mp_track_periods: a period's grid differs from the group's");
    }
    for (int p = 0; p + 1 < n_periods; ++p) {
        if (!std::isfinite(t_end[p])) return fail(MP_ERR_NONFINITE, "mp_track_periods: non-finite period end");
        if (p > 0 && t_end[p] < t_end[p - 1]) return fail(MP_ERR_INVALID_ARG, "mp_track_periods: ends not ascending");
    }
    MP_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Request* r = nullptr;
    mp::Req hr;
    unsigned modes = 0;
    int rc = prepare_request(ctx, g, o, s, &r, &hr, &modes);
    if (rc != MP_OK) return rc;
    r->fields.assign(fields, fields + n_periods);
    // the periods advance a request-owned copy of the group's state
    char* scratch = nullptr;
    if (cudaMallocAsync(&scratch, g->bytes, s) != cudaSuccess) {
        cudaGetLastError();
        drop_request(r);
        return fail(MP_ERR_OOM, "mp_track_periods: device allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(scratch, g->buf, g->bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        cudaFreeAsync(scratch, s);
        drop_request(r);
        return cuda_fail(e, "mp_track_periods: state copy");
    }
    const DevState sd = rebase(g->d, g->buf, scratch);
    const double t_stop = hr.p.t_stop;
    for (int p = 0; p < n_periods; ++p) {
        const bool last = p == n_periods - 1;
        mp::Req h = hr;
        h.in = sd;
        h.p.t_stop = last ? t_stop : std::min(t_stop, t_end[p]);
        split_ff(h.p.t_stop, h.p.tstop_hi, h.p.tstop_lo);
        h.p.update_group = 1;
        h.p.cont = p > 0;
        h.p.last = last ? 1 : 0;
        int sched = 0, blk = 0, spf = 0;
        resolve_launch(ctx, fields[p], o->precision, (modes & mp::MODE_TS) != 0, *o, &sched, &blk, &spf);
        rc = launch_requests(fields[p], &r, &h, 1, o->precision, sched, blk, spf, modes, s,
                             (p == 0 ? 1u : 0u) | (last ? 2u : 0u));
        if (rc != MP_OK) {
            cudaStreamSynchronize(s);
            cudaFreeAsync(scratch, s);
            drop_request(r);
            return rc;
        }
    }
    if (o->flags & MP_TRACK_UPDATE_GROUP) {
        e = cudaMemcpyAsync(g->buf, scratch, g->bytes, cudaMemcpyDeviceToDevice, s);
        g->field = fields[n_periods - 1];
    }
    cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        drop_request(r);
        return cuda_fail(e, "mp_track_periods: state copy");
    }
    *out = register_request(ctx, r);
    return MP_OK;
}

int mp_query(mp_ctx* ctx, mp_req id)
{
    if (!ctx) return fail(MP_ERR_INVALID_ARG, "mp_query: NULL");
    Request* r = find_req(ctx, id);
    if (!r) return fail(MP_ERR_NOT_READY, "mp_query: unknown request");
    cudaError_t e = cudaEventQuery(r->k1);
    if (e == cudaSuccess) return 1;
    if (e == cudaErrorNotReady) return 0;
    return cuda_fail(e, "mp_query");
}

int mp_wait(mp_ctx* ctx, mp_req id, int64_t timeout_us)
{
    if (!ctx) return fail(MP_ERR_INVALID_ARG, "mp_wait: NULL");
    Request* r = find_req(ctx, id);
    if (!r) return fail(MP_ERR_NOT_READY, "mp_wait: unknown request");
    return wait_event(r->k1, timeout_us);
}

namespace {

int copy_out(void* dst, const void* src, size_t bytes, bool dev, cudaStream_t s)
{
    if (!dst || bytes == 0) return MP_OK;
    if (dev) {
        MP_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s), "copy out");
    } else {
        MP_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost), "copy out");
    }
    return MP_OK;
}

int prepare_read(mp_ctx* ctx, Request* r, uint32_t flags, cudaStream_t s)
{
    if (flags & MP_DEVICE_PTR) {
        MP_CUDA(cudaStreamWaitEvent(s, r->k1, 0), "cudaStreamWaitEvent");
        return MP_OK;
    }
    int rc = wait_event(r->k1, -1);
    if (rc != MP_OK) return rc;
    unsigned long long h[N_COUNTERS];
    rc = read_counters(r, h);
    if (rc != MP_OK) return rc;
    if (h[COUNTER_ERR]) return fail(MP_ERR_DEVICE, "tracking kernel raised its error flag");
    (void)ctx;
    return MP_OK;
}

}  // namespace

int mp_get_endpoints(mp_ctx* ctx, mp_req id, const mp_endpoints* out, uint32_t flags, void* stream)
{
    if (!ctx || !out) return fail(MP_ERR_INVALID_ARG, "mp_get_endpoints: NULL");
    Request* r = find_req(ctx, id);
    if (!r) return fail(MP_ERR_NOT_READY, "mp_get_endpoints: unknown request");
    cudaSetDevice(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int rc = prepare_read(ctx, r, flags, s);
    if (rc != MP_OK) return rc;
    const bool dev = (flags & MP_DEVICE_PTR) != 0;
    const size_t n = (size_t)r->n;
    if ((rc = copy_out(out->cell, r->d.cell, 4 * n, dev, s)) != MP_OK) return rc;
    if ((rc = copy_out(out->x, r->d.x, 8 * n, dev, s)) != MP_OK) return rc;
    if ((rc = copy_out(out->y, r->d.y, 8 * n, dev, s)) != MP_OK) return rc;
    if ((rc = copy_out(out->z, r->d.z, 8 * n, dev, s)) != MP_OK) return rc;
    if ((rc = copy_out(out->px, r->d.px, 8 * n, dev, s)) != MP_OK) return rc;
    if ((rc = copy_out(out->py, r->d.py, 8 * n, dev, s)) != MP_OK) return rc;
    if ((rc = copy_out(out->pz, r->d.pz, 8 * n, dev, s)) != MP_OK) return rc;
    if ((rc = copy_out(out->t, r->d.t, 8 * n, dev, s)) != MP_OK) return rc;
    if ((rc = copy_out(out->status, r->d.status, n, dev, s)) != MP_OK) return rc;
    if ((rc = copy_out(out->steps, r->d.steps, 4 * n, dev, s)) != MP_OK) return rc;
    if ((rc = copy_out(out->exit_face, r->d.exit_face, n, dev, s)) != MP_OK) return rc;
    if ((rc = copy_out(out->hash, r->d.hash, 8 * n, dev, s)) != MP_OK) return rc;
    return MP_OK;
}

int mp_get_timeseries(mp_ctx* ctx, mp_req id, mp_ts_record* out, uint32_t flags, void* stream)
{
    if (!ctx || !out) return fail(MP_ERR_INVALID_ARG, "mp_get_timeseries: NULL");
    Request* r = find_req(ctx, id);
    if (!r) return fail(MP_ERR_NOT_READY, "mp_get_timeseries: unknown request");
    if (!r->d.ts) return fail(MP_ERR_INVALID_ARG, "mp_get_timeseries: request has no timeseries");
    cudaSetDevice(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int rc = prepare_read(ctx, r, flags, s);
    if (rc != MP_OK) return rc;
    return copy_out(out, r->d.ts, sizeof(mp_ts_record) * (size_t)r->n_times * (size_t)r->n,
                    (flags & MP_DEVICE_PTR) != 0, s);
}

int mp_get_pathlines(mp_ctx* ctx, mp_req id, mp_path_record* out, int64_t max_points, int64_t* n_points,
                     uint32_t flags, void* stream)
{
    if (!ctx || !n_points || max_points < 0 || (max_points > 0 && !out))
        return fail(MP_ERR_INVALID_ARG, "mp_get_pathlines: bad argument");
    Request* r = find_req(ctx, id);
    if (!r) return fail(MP_ERR_NOT_READY, "mp_get_pathlines: unknown request");
    if (!r->d.path) return fail(MP_ERR_INVALID_ARG, "mp_get_pathlines: request has no pathlines");
    cudaSetDevice(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int rc = wait_event(r->k1, -1);
    if (rc != MP_OK) return rc;
    unsigned long long h[N_COUNTERS];
    rc = read_counters(r, h);
    if (rc != MP_OK) return rc;
    if (h[COUNTER_ERR]) return fail(MP_ERR_DEVICE, "tracking kernel raised its error flag");
    const long long kept = std::min<long long>((long long)h[COUNTER_PATH], r->d.path_cap);
    const long long n = std::min<long long>(kept, max_points);
    *n_points = n;
    return copy_out(out, r->d.path, sizeof(mp_path_record) * (size_t)n, (flags & MP_DEVICE_PTR) != 0, s);
}

int mp_endpoints_device(mp_ctx* ctx, mp_req id, mp_endpoints* out, mp_ts_record** ts)
{
    if (!ctx) return fail(MP_ERR_INVALID_ARG, "mp_endpoints_device: NULL");
    Request* r = find_req(ctx, id);
    if (!r) return fail(MP_ERR_NOT_READY, "mp_endpoints_device: unknown request");
    if (out) {
        out->cell = r->d.cell;
        out->x = r->d.x; out->y = r->d.y; out->z = r->d.z;
        out->px = r->d.px; out->py = r->d.py; out->pz = r->d.pz;
        out->t = r->d.t;
        out->status = r->d.status;
        out->steps = r->d.steps;
        out->exit_face = r->d.exit_face;
        out->hash = reinterpret_cast<uint64_t*>(r->d.hash);
    }
    if (ts) *ts = r->d.ts;
    return MP_OK;
}

int mp_get_stats(mp_ctx* ctx, mp_req id, mp_stats* out)
{
    if (!ctx || !out) return fail(MP_ERR_INVALID_ARG, "mp_get_stats: NULL");
    Request* r = find_req(ctx, id);
    if (!r) return fail(MP_ERR_NOT_READY, "mp_get_stats: unknown request");
    cudaSetDevice(ctx->device);
    int rc = wait_event(r->k1, -1);
    if (rc != MP_OK) return rc;
    unsigned long long h[N_COUNTERS];
    rc = read_counters(r, h);
    if (rc != MP_OK) return rc;
    mp_stats st{};
    st.cell_steps = h[COUNTER_STEPS];
    for (int k = 0; k < MP_N_STATUS; ++k) st.n_status[k] = h[COUNTER_STATUS + k];
    float ms = 0.f;
    MP_CUDA(cudaEventElapsedTime(&ms, r->k0, r->k1), "cudaEventElapsedTime");
    st.kernel_ms = ms;
    st.device_error = h[COUNTER_ERR] ? 1 : 0;
    st.path_points = h[COUNTER_PATH];
    st.t_begin_ns = h[COUNTER_T_BEGIN] ? ~h[COUNTER_T_BEGIN] : 0ULL;
    st.t_end_ns = h[COUNTER_T_END];
    *out = st;
    return MP_OK;
}

int mp_req_free(mp_ctx* ctx, mp_req id)
{
    if (!ctx) return fail(MP_ERR_INVALID_ARG, "mp_req_free: NULL");
    Request* r = nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->reqs.find(id);
        if (it == ctx->reqs.end()) return fail(MP_ERR_NOT_READY, "mp_req_free: unknown request");
        r = it->second;
        if (r->graph_owned) return fail(MP_ERR_INVALID_ARG, "mp_req_free: the request belongs to a graph");
        ctx->reqs.erase(it);
    }
    cudaSetDevice(ctx->device);
    cudaFreeAsync(r->buf, r->stream);
    cudaEventDestroy(r->k0);
    cudaEventDestroy(r->k1);
    delete r;
    return MP_OK;
}

int mp_track_host(mp_ctx* ctx, const mp_field* f, int64_t n, const int32_t* cell, const double* local,
                  const double* t0, const mp_track_opts* o, int32_t n_chunks, const mp_endpoints* ep,
                  mp_ts_record* ts, mp_stats* stats)
{
    if (!ctx || !f || !o || !ep || n < 0) return fail(MP_ERR_INVALID_ARG, "mp_track_host: bad argument");
    if (n > 0 && (!cell || !local)) return fail(MP_ERR_INVALID_ARG, "mp_track_host: NULL cell/local");
    if (o->mode & MP_MODE_PATHLINE) return fail(MP_ERR_INVALID_ARG, "mp_track_host: pathline mode not supported");
    const bool want_ts = (o->mode & MP_MODE_TIMESERIES) != 0 && ts != nullptr;
    if (stats) *stats = mp_stats{};
    if (n == 0) return MP_OK;
    MP_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    // chunks of about 128 K particles (2 to 16 of them) unless the caller says
    long long nc = n_chunks > 0 ? n_chunks : std::min<long long>(16, std::max<long long>(2, (n + 131071) / 131072));
    nc = std::min<long long>(nc, n);
    const long long m = (n + nc - 1) / nc;
    nc = (n + m - 1) / m;
    // MP_SCHED_AUTO: the static schedule, whose blocks retire as their
    // particles finish so that the next chunk's blocks fill the SMs (the
    // persistent schedule holds its blocks until its queue drains)
    mp_track_opts oc = *o;
    if (oc.schedule == MP_SCHED_AUTO) oc.schedule = MP_SCHED_STATIC;

    // the context's two streams, kept across calls so that the chunks'
    // buffers are reused in stream order from the memory pool
    std::lock_guard<std::mutex> host_lk(ctx->host_mu);
    cudaEvent_t ev_start = nullptr, ev_join = nullptr, ev_end = nullptr;
    std::vector<mp_group*> groups;
    std::vector<mp_req> ids;
    int rc = MP_OK;
    auto cu = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && rc == MP_OK) rc = cuda_fail(e, what);
        return rc == MP_OK;
    };
    for (cudaStream_t& x : ctx->host_st)
        if (!x) cu(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking), "mp_track_host: stream");
    cudaStream_t* st = ctx->host_st;
    (rc == MP_OK) && cu(cudaEventCreate(&ev_start), "mp_track_host: event") &&
        cu(cudaEventCreate(&ev_join), "mp_track_host: event") && cu(cudaEventCreate(&ev_end), "mp_track_host: event") &&
        cu(cudaEventRecord(ev_start, st[0]), "mp_track_host: event") &&
        cu(cudaStreamWaitEvent(st[1], ev_start, 0), "mp_track_host: event");
    for (long long c = 0; c < nc && rc == MP_OK; ++c) {
        const long long off = c * m, cnt = std::min<long long>(m, n - off);
        cudaStream_t s = st[c & 1];
        mp_release_desc rd{};
        rd.n = cnt;
        rd.kind = MP_RELEASE_EXPLICIT;
        rd.flags = 0;
        rd.cell = cell + off;
        rd.local = local + 3 * off;
        rd.t0 = t0 ? t0 + off : nullptr;
        mp_group* g = nullptr;
        if ((rc = mp_release_group(ctx, f, &rd, s, &g)) != MP_OK) break;
        groups.push_back(g);
        mp_req id = 0;
        if ((rc = mp_track(ctx, g, &oc, s, &id)) != MP_OK) break;
        ids.push_back(id);
        Request* r = find_req(ctx, id);
        const size_t u = (size_t)cnt, q = (size_t)off;
        struct { void* dst; const void* src; size_t bytes; } cp[] = {
            {ep->cell ? ep->cell + q : nullptr, r->d.cell, 4 * u},
            {ep->x ? ep->x + q : nullptr, r->d.x, 8 * u},
            {ep->y ? ep->y + q : nullptr, r->d.y, 8 * u},
            {ep->z ? ep->z + q : nullptr, r->d.z, 8 * u},
            {ep->px ? ep->px + q : nullptr, r->d.px, 8 * u},
            {ep->py ? ep->py + q : nullptr, r->d.py, 8 * u},
            {ep->pz ? ep->pz + q : nullptr, r->d.pz, 8 * u},
            {ep->t ? ep->t + q : nullptr, r->d.t, 8 * u},
            {ep->status ? ep->status + q : nullptr, r->d.status, u},
            {ep->steps ? ep->steps + q : nullptr, r->d.steps, 4 * u},
            {ep->exit_face ? ep->exit_face + q : nullptr, r->d.exit_face, u},
            {ep->hash ? ep->hash + q : nullptr, r->d.hash, 8 * u},
        };
        for (auto& x : cp)
            if (x.dst && !cu(cudaMemcpyAsync(x.dst, x.src, x.bytes, cudaMemcpyDeviceToHost, s), "mp_track_host: copy"))
                break;
        if (rc == MP_OK && want_ts && r->d.ts && r->n_times > 0)
            cu(cudaMemcpy2DAsync(ts + q, sizeof(mp_ts_record) * (size_t)n, r->d.ts, sizeof(mp_ts_record) * u,
                                 sizeof(mp_ts_record) * u, (size_t)r->n_times, cudaMemcpyDeviceToHost, s),
               "mp_track_host: timeseries copy");
    }
    // join the streams, then wait (bounded) for the last copy
    if (st[0] && st[1] && ev_join && ev_end) {
        cudaError_t e = cudaEventRecord(ev_join, st[1]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st[0], ev_join, 0);
        if (e == cudaSuccess) e = cudaEventRecord(ev_end, st[0]);
        if (e == cudaSuccess) {
            const int w = wait_event(ev_end, -1);
            if (w != MP_OK && rc == MP_OK) rc = w;
        } else {
            cu(e, "mp_track_host: join");
            cudaStreamSynchronize(st[0]);
            cudaStreamSynchronize(st[1]);
        }
    }
    mp_stats sum{};
    for (mp_req id : ids) {
        mp_stats one{};
        const int g = mp_get_stats(ctx, id, &one);
        if (g != MP_OK) {
            if (rc == MP_OK) rc = g;
            continue;
        }
        sum.cell_steps += one.cell_steps;
        for (int k = 0; k < MP_N_STATUS; ++k) sum.n_status[k] += one.n_status[k];
        sum.device_error |= one.device_error;
        if (one.t_begin_ns && (!sum.t_begin_ns || one.t_begin_ns < sum.t_begin_ns)) sum.t_begin_ns = one.t_begin_ns;
        if (one.t_end_ns > sum.t_end_ns) sum.t_end_ns = one.t_end_ns;
    }
    if (rc == MP_OK && sum.device_error) rc = fail(MP_ERR_DEVICE, "mp_track_host: tracking kernel raised its error flag");
    if (ev_start && ev_end && rc == MP_OK) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev_start, ev_end) == cudaSuccess) sum.kernel_ms = ms;
    }
    if (stats) *stats = sum;
    for (mp_req id : ids) mp_req_free(ctx, id);
    for (mp_group* g : groups) mp_group_free(g);
    if (st[0]) cudaStreamSynchronize(st[0]);
    if (st[1]) cudaStreamSynchronize(st[1]);
    for (cudaEvent_t e : {ev_start, ev_join, ev_end})
        if (e) cudaEventDestroy(e);
    return rc;
}

}  // extern "C"

namespace mp {

void set_last_error(const char* msg) { g_err = msg ? msg : ""; }

const DevField* field_device_view(const mp_field* f) { return &f->d; }
bool field_is_usg(const mp_field* f) { return f->usg != 0; }
int field_device(const mp_field* f) { return f->ctx->device; }

}  // namespace mp

extern "C" {

int mp_set_tuning(mp_ctx* ctx, const mp_field* f, int32_t precision, int32_t timeseries, const mp_tuning* t)
{
    if (!ctx || !f || !t) return fail(MP_ERR_INVALID_ARG, "mp_set_tuning: NULL");
    if ((t->schedule != MP_SCHED_STATIC && t->schedule != MP_SCHED_DYNAMIC) || t->block < 32 || t->block > 256 ||
        t->steps_per_fetch < 0)
        return fail(MP_ERR_INVALID_ARG, "mp_set_tuning: bad configuration");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->tuned[TuneKey{f, precision, timeseries ? 1 : 0}] = *t;
    return MP_OK;
}

int mp_autotune(mp_ctx* ctx, mp_group* g, const mp_track_opts* o, int64_t sample, void* stream, mp_tuning* out)
{
    if (!ctx || !g || !o || !out) return fail(MP_ERR_INVALID_ARG, "mp_autotune: NULL argument");
    MP_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    struct Cand { int sched, block, spf; };
    std::vector<Cand> cands;
    for (int b : {64, 128, 256}) cands.push_back({MP_SCHED_STATIC, b, 0});
    for (int b : {64, 128, 256})
        for (int spf : {1, 4, 16}) cands.push_back({MP_SCHED_DYNAMIC, b, spf});
    mp_track_opts oo = *o;
    oo.flags &= ~MP_TRACK_UPDATE_GROUP;
    oo.schedule = MP_SCHED_DYNAMIC;
    mp_tuning best{};
    best.ms = INFINITY;
    unsigned modes = 0;
    for (size_t ci = 0; ci <= cands.size(); ++ci) {
        // the first pass warms the field and the allocator and is not counted
        const Cand c = ci == 0 ? cands[0] : cands[ci - 1];
        Request* r = nullptr;
        mp::Req hr;
        int rc = prepare_request(ctx, g, &oo, s, &r, &hr, &modes);
        if (rc != MP_OK) return rc;
        if (sample > 0 && hr.p.n > sample) hr.p.n = sample;
        rc = launch_requests(g->field, &r, &hr, 1, o->precision, c.sched, c.block, c.spf, modes, s);
        if (rc == MP_OK) rc = wait_event(r->k1, -1);
        float ms = 0.f;
        if (rc == MP_OK && cudaEventElapsedTime(&ms, r->k0, r->k1) != cudaSuccess) rc = fail(MP_ERR_CUDA, "timing");
        drop_request(r);
        if (rc != MP_OK) return rc;
        if (ci > 0 && ms < best.ms) {
            best.ms = ms;
            best.schedule = c.sched;
            best.block = c.block;
            best.steps_per_fetch = c.spf;
        }
    }
    best.tried = (int32_t)cands.size();
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->tuned[TuneKey{g->field, o->precision, (modes & mp::MODE_TS) ? 1 : 0}] = best;
    }
    *out = best;
    return MP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Captured batches: release + tracking of a fixed set of box-release
// requests as one CUDA graph, replayed with new release descriptors.
// ---------------------------------------------------------------------------

struct mp_graph {
    mp_ctx* ctx = nullptr;
    const mp_field* field = nullptr;
    std::vector<mp_group*> groups;          // views into state
    std::vector<Request*> reqs;
    std::vector<mp_req> ids;
    std::vector<mp::BoxRelease> desc;       // host copy of the device descriptors
    char* state = nullptr;                  // every group's state arrays
    char* tables = nullptr;                 // descriptors, starts, batch tables, queues
    mp::BoxRelease* d_desc = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t k0 = nullptr, k1 = nullptr;
};

namespace {

int graph_release_check(const mp_release_desc& r)
{
    if (r.kind != MP_RELEASE_BOX) return fail(MP_ERR_INVALID_ARG, "mp_graph: only box releases can be captured");
    if (r.n < 0) return fail(MP_ERR_INVALID_ARG, "mp_graph: n < 0");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(r.lo[a]) || !std::isfinite(r.hi[a]) || r.hi[a] < r.lo[a])
            return fail(MP_ERR_INVALID_ARG, "mp_graph: box must be finite with lo <= hi");
    return MP_OK;
}

void graph_destroy(mp_graph* G)
{
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    for (Request* r : G->reqs) drop_request(r);
    for (mp_group* g : G->groups) delete g;
    if (G->state) cudaFree(G->state);
    if (G->tables) cudaFree(G->tables);
    if (G->k0) cudaEventDestroy(G->k0);
    if (G->k1) cudaEventDestroy(G->k1);
    delete G;
}

}  // namespace

extern "C" {

int mp_graph_create(mp_ctx* ctx, const mp_field* f, int n_reqs, const mp_release_desc* rel,
                    const mp_track_opts* opts, void* stream, mp_graph** out)
{
    if (!ctx || !f || !rel || !opts || !out || n_reqs < 1) return fail(MP_ERR_INVALID_ARG, "mp_graph_create: bad argument");
    if (n_reqs >= (1 << 24)) return fail(MP_ERR_INVALID_ARG, "mp_graph_create: more than 2^24 - 1 requests");
    if (f->ctx != ctx) return fail(MP_ERR_INVALID_ARG, "mp_graph_create: field of another context");
    if (f->usg) return fail(MP_ERR_INVALID_ARG, "mp_graph_create: box releases need a rectilinear grid");
    for (int i = 0; i < n_reqs; ++i) {
        const int rc = graph_release_check(rel[i]);
        if (rc != MP_OK) return rc;
        if (opts[i].flags & MP_TRACK_UPDATE_GROUP)
            return fail(MP_ERR_INVALID_ARG, "mp_graph_create: a replayed release makes MP_TRACK_UPDATE_GROUP moot");
        if (opts[i].precision != MP_PREC_FP64 && opts[i].precision != MP_PREC_MIXED)
            return fail(MP_ERR_INVALID_ARG, "mp_graph_create: precision must be MP_PREC_FP64 or MP_PREC_MIXED");
    }
    MP_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    mp_graph* G = new mp_graph();
    G->ctx = ctx;
    G->field = f;
    auto bail = [&](int rc) { cudaStreamSynchronize(s); graph_destroy(G); return rc; };
    // group state of every request in one allocation
    std::vector<size_t> goff((size_t)n_reqs + 1, 0);
    for (int i = 0; i < n_reqs; ++i) goff[i + 1] = goff[i] + align256(group_bytes(rel[i].n));
    if (cudaMalloc(&G->state, goff[n_reqs]) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(MP_ERR_OOM, "mp_graph_create: device allocation failed"));
    }
    std::vector<long long> starts((size_t)n_reqs + 1, 0);
    std::vector<mp::Req> hr((size_t)n_reqs);
    std::vector<unsigned> md((size_t)n_reqs, 0);
    for (int i = 0; i < n_reqs; ++i) {
        mp_group* g = new mp_group();
        g->ctx = ctx;
        g->field = f;
        g->n = rel[i].n;
        g->buf = G->state + goff[i];
        g->bytes = group_bytes(rel[i].n);
        g->stream = s;
        g->d = group_view(G->state + goff[i], rel[i].n);
        G->groups.push_back(g);
        Request* r = nullptr;
        const int rc = prepare_request(ctx, g, &opts[i], s, &r, &hr[i], &md[i]);
        if (rc != MP_OK) return bail(rc);
        r->graph_owned = true;
        cudaEventDestroy(r->k0);
        cudaEventDestroy(r->k1);
        r->k0 = r->k1 = nullptr;
        G->reqs.push_back(r);
        starts[i + 1] = starts[i] + rel[i].n;
        mp::BoxRelease b{};
        b.st = g->d;
        b.n = rel[i].n;
        for (int a = 0; a < 3; ++a) { b.lo[a] = rel[i].lo[a]; b.hi[a] = rel[i].hi[a]; }
        b.seed = rel[i].seed;
        b.id_offset = rel[i].id_offset;
        G->desc.push_back(b);
    }
    if (cudaEventCreate(&G->k0) != cudaSuccess || cudaEventCreate(&G->k1) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "mp_graph_create: events"));
    for (Request* r : G->reqs) { r->k0 = G->k0; r->k1 = G->k1; }
    // device tables: release descriptors and starts, then per precision the
    // tracking batch (request table, its starts, queue head)
    std::vector<int> sel[2];
    for (int i = 0; i < n_reqs; ++i) sel[opts[i].precision == MP_PREC_FP64 ? 0 : 1].push_back(i);
    size_t off = 0;
    const size_t o_desc = off; off = align256(off + sizeof(mp::BoxRelease) * (size_t)n_reqs);
    const size_t o_st = off; off = align256(off + sizeof(long long) * ((size_t)n_reqs + 1));
    size_t o_req[2], o_bst[2], o_q[2];
    for (int p = 0; p < 2; ++p) {
        o_req[p] = off; off = align256(off + sizeof(mp::Req) * sel[p].size());
        o_bst[p] = off; off = align256(off + sizeof(long long) * (sel[p].size() + 1));
        o_q[p] = off; off = align256(off + sizeof(unsigned long long));
    }
    if (cudaMalloc(&G->tables, off) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(MP_ERR_OOM, "mp_graph_create: device allocation failed"));
    }
    G->d_desc = reinterpret_cast<mp::BoxRelease*>(G->tables + o_desc);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess)
        e = cudaMemcpy(G->d_desc, G->desc.data(), sizeof(mp::BoxRelease) * (size_t)n_reqs, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(G->tables + o_st, starts.data(), sizeof(long long) * ((size_t)n_reqs + 1),
                       cudaMemcpyHostToDevice);
    mp::Batch bat[2]{};
    unsigned modes[2] = {0u, 0u};
    for (int p = 0; p < 2 && e == cudaSuccess; ++p) {
        std::vector<mp::Req> rq;
        std::vector<long long> bs(1, 0);
        for (int i : sel[p]) {
            rq.push_back(hr[i]);
            bs.push_back(bs.back() + rel[i].n);
            modes[p] |= md[i];
        }
        if (!rq.empty())
            e = cudaMemcpy(G->tables + o_req[p], rq.data(), sizeof(mp::Req) * rq.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !rq.empty())
            e = cudaMemcpy(G->tables + o_bst[p], bs.data(), sizeof(long long) * bs.size(), cudaMemcpyHostToDevice);
        bat[p].reqs = reinterpret_cast<const mp::Req*>(G->tables + o_req[p]);
        bat[p].starts = reinterpret_cast<const long long*>(G->tables + o_bst[p]);
        bat[p].n_reqs = (int)sel[p].size();
        bat[p].n_total = bs.back();
        bat[p].queue = reinterpret_cast<unsigned long long*>(G->tables + o_q[p]);
    }
    if (e != cudaSuccess) return bail(cuda_fail(e, "mp_graph_create: tables"));
    // capture: clear counters and queue heads, release, track
    const mp::DevField& fd = *mp::field_device_view(f);
    cudaStream_t cs = nullptr;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(cuda_fail(e, "mp_graph_create: stream"));
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    for (Request* r : G->reqs)
        if (e == cudaSuccess) e = cudaMemsetAsync(r->d.counters, 0, sizeof(unsigned long long) * N_COUNTERS, cs);
    for (int p = 0; p < 2 && e == cudaSuccess; ++p)
        if (!sel[p].empty()) e = cudaMemsetAsync(bat[p].queue, 0, sizeof(unsigned long long), cs);
    if (e == cudaSuccess)
        e = mp::launch_release_boxes(fd, G->d_desc, reinterpret_cast<const long long*>(G->tables + o_st), n_reqs,
                                     starts[n_reqs], cs);
    for (int p = 0; p < 2 && e == cudaSuccess; ++p) {
        if (sel[p].empty()) continue;
        const int prec = p == 0 ? MP_PREC_FP64 : MP_PREC_MIXED;
        int sched = 0, blk = 0, spf = 0;
        resolve_launch(ctx, f, prec, (modes[p] & mp::MODE_TS) != 0, opts[sel[p][0]], &sched, &blk, &spf);
        bat[p].steps_per_fetch = spf > 0 ? spf : 4;
        e = prec == MP_PREC_FP64 ? mp::launch_track_fp64(fd, bat[p], modes[p], sched, blk > 0 ? blk : 128, 0, cs)
                                 : mp::launch_track_mixed(fd, bat[p], modes[p], sched, blk > 0 ? blk : 128, 0, cs);
        if (e == cudaSuccess) e = mp::launch_spread_window(bat[p], cs);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    G->graph = graph;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&G->exec, G->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return bail(cuda_fail(e, "mp_graph_create: capture"));
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (Request* r : G->reqs) {
            const int64_t id = ctx->next_id++;
            ctx->reqs[id] = r;
            G->ids.push_back(id);
        }
        ctx->graphs.insert(G);
    }
    *out = G;
    return MP_OK;
}

int mp_graph_set_release(mp_graph* G, int i, const mp_release_desc* rel, void* stream)
{
    if (!G || !rel || i < 0 || i >= (int)G->desc.size()) return fail(MP_ERR_INVALID_ARG, "mp_graph_set_release: bad argument");
    int rc = graph_release_check(*rel);
    if (rc != MP_OK) return rc;
    if (rel->n != G->desc[i].n) return fail(MP_ERR_SHAPE, "mp_graph_set_release: the particle count is fixed");
    MP_CUDA(cudaSetDevice(G->ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    mp::BoxRelease& b = G->desc[i];
    for (int a = 0; a < 3; ++a) { b.lo[a] = rel->lo[a]; b.hi[a] = rel->hi[a]; }
    b.seed = rel->seed;
    b.id_offset = rel->id_offset;
    // ordered after earlier work on the stream; synchronous so that the host
    // copy may change again at once
    cudaError_t e = cudaMemcpyAsync(G->d_desc + i, &b, sizeof(mp::BoxRelease), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "mp_graph_set_release");
    return MP_OK;
}

int mp_graph_launch(mp_graph* G, void* stream)
{
    if (!G) return fail(MP_ERR_INVALID_ARG, "mp_graph_launch: NULL");
    MP_CUDA(cudaSetDevice(G->ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaEventRecord(G->k0, s);
    if (e == cudaSuccess) e = cudaGraphLaunch(G->exec, s);
    if (e == cudaSuccess) e = cudaEventRecord(G->k1, s);
    if (e != cudaSuccess) return cuda_fail(e, "mp_graph_launch");
    for (Request* r : G->reqs) r->stream = s;
    return MP_OK;
}

int mp_graph_requests(const mp_graph* G, mp_req* ids)
{
    if (!G || !ids) return fail(MP_ERR_INVALID_ARG, "mp_graph_requests: NULL");
    for (size_t i = 0; i < G->ids.size(); ++i) ids[i] = G->ids[i];
    return MP_OK;
}

int mp_graph_free(mp_graph* G)
{
    if (!G) return fail(MP_ERR_INVALID_ARG, "mp_graph_free: NULL");
    mp_ctx* ctx = G->ctx;
    cudaSetDevice(ctx->device);
    int rc = wait_event(G->k1, -1);
    if (rc != MP_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (mp_req id : G->ids) ctx->reqs.erase(id);
        ctx->graphs.erase(G);
    }
    graph_destroy(G);
    return MP_OK;
}

}  // extern "C"
