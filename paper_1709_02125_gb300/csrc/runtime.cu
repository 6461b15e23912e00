// Executor and C ABI of liboc: dataset stores, the lazy loop queue, plan selection,
// and the three-stream tile pipeline.
//
// arXiv 1709.02125, Sec. 3 (lazy loop chains, data owned by the library), Sec. 4,
// Algorithm 1 (explicitly managed tiling with three streams) and Sec. 4.1 (copy
// avoidance, cyclic option, speculative prefetch).
//
// Pipeline. With upload lookahead k = depth - 2, phase p (p = -k .. T) uploads tile
// p + k on stream 1, computes tile p on stream 0 and downloads tile p - 1 on stream
// 2. A slab row is live from the phase of its upload (or of its first tile, if it is
// not uploaded) to the phase of its download (or of its last tile). Slabs are sized
// (analysis.cpp) so that rows live in the same phase never share a slot; an
// operation of phase p that overwrites slots therefore only has to wait for the
// operations of phases <= p - 1 on the other streams:
//   upload  (phase p): waits compute(p - 1) and download of tile p - 2;
//   compute (tile p) : waits upload(p) and download of tile p - 2;
//   download(tile p) : waits compute(p).
// Rows shared by consecutive tiles stay in their slot, which replaces the paper's
// right-edge to left-edge copy between slots (Algorithm 1, finishing phase).
// The loops of one tile run on stream 0 and, where independent of their neighbours,
// on a second compute stream that is joined back before the tile's end event. The
// compute streams carry kernels only: the parameter block goes up on stream 1 and the
// reduction results come back on stream 2. A repeated chain is captured once as one
// CUDA graph over all streams and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <array>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <sys/syscall.h>
#include <thread>
#include <unistd.h>
#include <unordered_map>
#include <vector>

#include "../../include/oc.h"
#include "launch.h"
#include "oc_internal.h"
#include "physics.h"
#include "mlp.h"
#include "planner.h"

namespace oc {

static char g_err[1024] = "";

static int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define OC_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(OC_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                              \
    } while (0)

// One profiled launch: events bracketing it on the compute stream.
struct ProfRec {
    int kernel;
    int launches;         // consecutive launches of `kernel` between the two events
    double bytes, points;
    cudaEvent_t a, b;
};

struct KStat {
    long long launches = 0;
    double ms = 0, bytes = 0, points = 0;
};

struct GraphSet {
    std::vector<cudaGraphExec_t> tiles;
    std::vector<std::vector<ProfRec>> prof;  // events captured into each tile's graph
};

// The whole pipeline of one chain shape (parameter upload, every tile's uploads,
// kernels and downloads on the three streams with their dependencies, the reduction
// combine, the result read-back and the speculative prefetch) captured once as one
// CUDA graph, with what the capture counted.
struct ChainGraph {
    cudaGraphExec_t exec = nullptr;
    double h2d = 0, d2h = 0, prefetched = 0;
    int launches = 0;
    bool pf_active = false;
    uint64_t pf_sig = 0;
    double pf_bytes = 0;
    std::vector<std::vector<Interval>> pf_rows;
    // pinned parameter / result staging the graph's copy nodes point at (owned)
    double* hp = nullptr;
    double* hr = nullptr;
};

struct Prefetch {
    bool active = false;
    uint64_t sig = 0;
    std::vector<std::vector<Interval>> rows;  // per plan dataset index
    double bytes = 0;
};

struct Ctx {
    uint32_t flags = 0;
    int planner_mode = OC_PLAN_FIXED;
    bool dryrun = false;
    long long budget = 0;
    char* arena = nullptr;
    long long arena_bytes = 0;
    bool own_arena = false;
    cudaStream_t st[3] = {nullptr, nullptr, nullptr};
    bool own_streams = false;
    // second compute stream for independent loops of one tile, and its events
    cudaStream_t s0b = nullptr;
    cudaEvent_t ev_tf = nullptr, ev_tj = nullptr;
    // side stream of the upload stream for the SM-driven halo-strip copies of a tile
    // (they run beside the copy engines' row copies instead of after them)
    cudaStream_t s1b = nullptr;
    cudaEvent_t ev_sf = nullptr, ev_sj = nullptr;
    std::vector<cudaEvent_t> ev_launch;
    std::vector<Dat> dats;
    std::vector<int> red_ops;
    std::vector<double> red_val;
    std::vector<char> red_has;
    std::vector<Loop> queue;
    std::unordered_map<uint64_t, Plan> plans;       // by plan signature
    std::unordered_map<uint64_t, Plan*> chosen;      // chain shape + settings -> plan
    std::unordered_map<uint64_t, std::vector<std::vector<LaunchDesc>>> descs;  // plan sig -> tiles
    std::unordered_map<uint64_t, GraphSet> graphs;
    std::unordered_map<uint64_t, ChainGraph> chain_graphs;
    cudaEvent_t ev_fork = nullptr, ev_fork2 = nullptr, ev_j1 = nullptr, ev_j2 = nullptr, ev_par = nullptr,
                ev_res = nullptr, ev_resup = nullptr;
    const Plan* last = nullptr;   // plan of the most recent flush (owned by `plans`)
    int force_h = 0, force_depth = 0;
    double force_res = -1.0;   // share of the budget for resident datasets; < 0: planner
    std::vector<cudaEvent_t> ev_up, ev_comp, ev_down;
    // 1 where the tile's upload / download issued at least one copy and its event was
    // recorded; an empty phase records nothing and nothing waits for it
    std::vector<char> up_rec, dn_rec;
    cudaEvent_t ev_pf = nullptr, ev_end = nullptr;
    double* h_params = nullptr;
    size_t h_params_cap = 0;
    double* h_results = nullptr;
    size_t h_results_cap = 0;
    Prefetch pf;
    bool resident_mode = false;
    long long resident_bytes = 0;
    double timeout_s = 600.0;
    oc_stats_t stats{};
    // profiling (OC_FLAG_PROFILE)
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_next = 0;
    std::vector<ProfRec> prof_pending;
    std::unordered_map<int, KStat> kstats;
    // tracing (OC_FLAG_TRACE)
    struct TraceRec { int tile, kind; cudaEvent_t a, b; double bytes; };
    std::vector<cudaEvent_t> tr_pool;
    size_t tr_next = 0;
    std::vector<TraceRec> tr;
    cudaEvent_t tr_t0 = nullptr;
    std::vector<oc_trace_rec> tr_out;
    // planner: features of the last planned chain, autotuner table (h, depth, ms, grid
    // index, largest fitting h) of the last autotuned chain
    float features[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    std::vector<std::array<double, 6>> tune;
    // host-side fault injection (oc_inject_fault): calls at site k still to pass before
    // the next one fails; -1 = disarmed
    long long fault_after[3] = {-1, -1, -1};
    // autotuning trials
    bool trial = false;
    cudaEvent_t tm0 = nullptr, tm1 = nullptr;   // timing events of a trial
    char* trial_sink = nullptr;                 // pinned scratch receiving trial downloads
    size_t trial_sink_bytes = 0;
};

static Ctx* g = nullptr;

// ---------------------------------------------------------------------------------
static int wait_event(cudaEvent_t ev, double timeout_s)
{
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return OC_OK;
        if (e != cudaErrorNotReady)
            return fail(OC_ERR_CUDA, "event wait failed: %s", cudaGetErrorString(e));
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_s) return fail(OC_ERR_TIMEOUT, "bounded wait expired after %.1f s", el);
        if (el > 1e-3) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// Injected fault at `site` (0 upload copy, 1 download copy, 2 kernel launch): true when
// the armed countdown reaches this call, which then fails without calling CUDA.
static bool injected(int site)
{
    long long& n = g->fault_after[site];
    if (n < 0) return false;
    if (n > 0) { --n; return false; }
    n = -1;
    return true;
}

static int wait_stream(cudaStream_t s)
{
    OC_CUDA(cudaEventRecord(g->ev_end, s));
    return wait_event(g->ev_end, g->timeout_s);
}

static int ensure_events(int T)
{
    while ((int)g->ev_up.size() < T) {
        cudaEvent_t a, b, c;
        OC_CUDA(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
        OC_CUDA(cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
        OC_CUDA(cudaEventCreateWithFlags(&c, cudaEventDisableTiming));
        g->ev_up.push_back(a);
        g->ev_comp.push_back(b);
        g->ev_down.push_back(c);
    }
    return OC_OK;
}

static void* host_alloc(size_t bytes, bool pinned)
{
    void* p = nullptr;
    if (pinned) {
        if (cudaHostAlloc(&p, bytes, cudaHostAllocPortable) != cudaSuccess) return nullptr;
        return p;
    }
    return malloc(bytes);
}

static void host_free(void* p, bool pinned)
{
    if (!p) return;
    if (pinned) cudaFreeHost(p);
    else free(p);
}

// ---------------------------------------------------------------------------------
// Copies between the pinned store and a slab. Rows [a, b) of dataset d go to slots
// (y - y0) mod S of the slab at `slab`; a range crossing the slab end is split.
// With x0 < x1 (uploads of rows first written over x in [x0, x1)) only the x columns
// outside [x0, x1) are copied: two strided copies over every x-line of the rows, added
// to `strips` (an SM-driven copy launched by the caller) when the host store is mapped,
// else issued to the copy engines.
static int flush_strips(StripBatch& sb, cudaStream_t s, oc_stats_t* S)
{
    if (sb.njobs == 0) return OC_OK;
    cudaError_t e = launch_strips(sb, s);
    if (e != cudaSuccess) return fail(OC_ERR_CUDA, "strip upload launch failed: %s", cudaGetErrorString(e));
    if (S) S->kernel_launches++;
    sb.njobs = 0;
    return OC_OK;
}

static int copy_rows(const Dat& d, char* slab, int S, int a, int b, bool up, cudaStream_t s,
                     double& bytes, int x0 = 0, int x1 = 0, char* host_override = nullptr,
                     StripBatch* strips = nullptr, oc_stats_t* stats = nullptr, cudaStream_t strip_s = nullptr)
{
    if (!strip_s) strip_s = s;
    const long long rb = d.row_bytes();
    const size_t lp = (size_t)d.pitch * d.esz;
    // the host store holds rows [y0, y0 + nrows) only: a row range outside it is a
    // planning error, reported before any copy touches memory outside the store
    if (!host_override && a < b && (a < d.y0 || b > d.y0 + d.nrows))
        return fail(OC_ERR_STATE, "%s copy of rows [%d, %d) outside the host store's rows [%d, %d)",
                    up ? "upload" : "download", a, b, d.y0, d.y0 + d.nrows);
    if (S <= 0 || (x0 < x1 && (x0 < -d.hlo[0] || x1 > d.size[0] + d.hhi[0])))
        return fail(OC_ERR_STATE, "copy of rows [%d, %d): slab of %d rows, columns [%d, %d)", a, b, S, x0, x1);
    while (a < b) {
        int slot = (int)(((long long)(a - d.y0)) % S);
        int n = std::min(b - a, S - slot);
        char* dev = slab + (long long)slot * rb;
        char* host = host_override ? host_override : (char*)d.host + (long long)(a - d.y0) * rb;
        if (x0 < x1) {
            const cudaMemcpyKind kind = up ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
            const size_t lines = (size_t)n * d.ylines;
            const long long c0 = d.ox - d.hlo[0];                       // first column (x = -hlo)
            const long long cl = (long long)x0 + d.hlo[0];              // left strip width
            const long long cr = (long long)d.size[0] + d.hhi[0] - x1;  // right strip width
            const long long c1 = d.ox + x1;
            char* dsts[2] = {up ? dev + c0 * d.esz : host + c0 * d.esz, up ? dev + c1 * d.esz : host + c1 * d.esz};
            const char* srcs[2] = {up ? host + c0 * d.esz : dev + c0 * d.esz, up ? host + c1 * d.esz : dev + c1 * d.esz};
            const long long w[2] = {cl, cr};
            const bool sm_copy = up && strips && d.host_dev && !host_override;
            for (int k = 0; k < 2; ++k)
                if (w[k] > 0) {
                    if (sm_copy) {
                        if (strips->njobs == kStripJobs) {
                            int r = flush_strips(*strips, strip_s, stats);
                            if (r) return r;
                        }
                        StripJob& j = strips->job[strips->njobs++];
                        j.src = d.host_dev + (srcs[k] - (const char*)d.host);
                        j.dst = dsts[k];
                        j.pitch = (long long)lp;
                        j.lines = (int)lines;
                        j.words = (int)(w[k] * d.esz / 4);
                    } else {
                        OC_CUDA(cudaMemcpy2DAsync(dsts[k], lp, srcs[k], lp, (size_t)w[k] * d.esz, lines, kind, s));
                    }
                    bytes += (double)w[k] * d.esz * lines;
                }
        } else {
            if (injected(up ? 0 : 1))
                return fail(OC_ERR_CUDA, "injected fault: %s copy of rows [%d, %d)", up ? "upload" : "download", a, a + n);
            if (up) OC_CUDA(cudaMemcpyAsync(dev, host, (size_t)n * rb, cudaMemcpyHostToDevice, s));
            else OC_CUDA(cudaMemcpyAsync(host, dev, (size_t)n * rb, cudaMemcpyDeviceToHost, s));
            bytes += (double)n * rb;
        }
        a += n;
    }
    return OC_OK;
}

// Subtract prefetched rows from an upload interval; emit the remainder.
template <typename F>
static int for_missing(const Interval& iv, const std::vector<Interval>* have, F emit)
{
    int a = iv.a;
    if (have) {
        for (const Interval& h : *have) {
            if (h.b <= a || h.a >= iv.b) continue;
            if (h.a > a) { int r = emit(a, h.a); if (r) return r; }
            a = std::max(a, h.b);
        }
    }
    if (a < iv.b) return emit(a, iv.b);
    return OC_OK;
}

// ---------------------------------------------------------------------------------
static DView make_view(const Dat& d, char* slab, int S, int W0)
{
    DView v;
    v.base = slab;
    v.row_elems = d.row_elems;
    v.pitch = d.pitch;
    v.ox = d.ox;
    v.oy = d.ndim == 3 ? d.hlo[1] : 0;
    v.S = S;
    if (W0 < d.y0) W0 = d.y0;
    v.W0 = W0;
    v.slot0 = (int)(((long long)(W0 - d.y0)) % S);
    v.nx = d.size[0];
    v.ny = d.ndim == 3 ? d.size[1] : 1;
    v.periodic = 0;
    if (d.periodic & 1) v.periodic |= 1;
    if (d.ndim == 3 && (d.periodic & 2)) v.periodic |= 2;
    v.pad_ = 0;
    return v;
}

static char* slab_base(const Plan& P, int di)
{
    const DatPlan& dp = P.dp[di];
    const Dat& d = g->dats[dp.dat];
    if (d.managed) return (char*)d.host;
    if (P.incore && d.resident) return g->arena + d.res_off;
    return g->arena + dp.off;
}

static long long scratch_base(const Plan& P)
{
    return P.incore ? g->resident_bytes : P.slab_bytes;
}

static void build_descs(const Plan& P, const std::vector<Loop>& loops,
                        std::vector<std::vector<LaunchDesc>>& out)
{
    out.assign(P.T, {});
    const long long sb = scratch_base(P);
    for (int t = 0; t < P.T; ++t)
        for (int i = 0; i < P.L; ++i) {
            int s = P.s(t, i), e = P.e(t, i);
            const Loop& lp = loops[i];
            if (s >= e || lp.points() == 0) continue;
            const int sa = lp.ndim - 1;
            LaunchDesc d;
            memset(&d, 0, sizeof(d));
            d.kernel = lp.kernel;
            d.ndim = lp.ndim;
            for (int a = 0; a < 3; ++a) { d.lo[a] = lp.lo[a]; d.hi[a] = lp.hi[a]; }
            d.lo[sa] = s;
            d.hi[sa] = e;
            d.nargs = (int)lp.args.size();
            d.dtype = -1;
            int ns = 0;
            for (int j = 0; j < d.nargs; ++j) {
                const Arg& ar = lp.args[j];
                d.access[j] = ar.access;
                d.npts[j] = (int)ar.off.size();
                if (ar.access == OC_REDUCE) continue;
                const Dat& dd = g->dats[ar.dat];
                if (d.dtype < 0) d.dtype = dd.dtype;
                int di = P.dat_index[ar.dat];
                int W0 = (ar.access == OC_READ || ar.access == OC_RW) ? s + ar.rmin[sa] : s;
                if (ar.access == OC_RW) W0 = std::min(W0, s);
                // a managed store is addressed in place: every row at its own slot
                d.v[j] = make_view(dd, slab_base(P, di), dd.managed ? dd.nrows : P.dp[di].S, W0);
                if (ar.access == OC_READ && j >= 1)
                    for (auto& o : ar.off) {
                        if (ns < kLaunchMaxSamples) {
                            d.sarg[ns] = j;
                            d.soff[ns][0] = o[0]; d.soff[ns][1] = o[1]; d.soff[ns][2] = o[2];
                        }
                        ++ns;
                    }
            }
            if (lp.kernel == OC_K_REDUCE) ns = 0;
            d.nsamp = ns;
            // lean addressing for LINCOMB / COPY: per-sample base pointers and first slots
            if ((lp.kernel == OC_K_LINCOMB || lp.kernel == OC_K_COPY) && ns <= kLaunchMaxSamples) {
                bool wrap = false;
                for (int j = 0; j < d.nargs; ++j)
                    if (lp.args[j].access != OC_REDUCE && d.v[j].periodic) wrap = true;
                if (!wrap) {
                    const long long esz = d.dtype == OC_F32 ? 4 : 8;
                    auto rec = [&](const DView& v, int dx, int dy, int ds) {
                        SampleRec r;
                        r.p0 = v.base + ((long long)(dy + v.oy) * v.pitch + v.ox + dx) * esz;
                        r.row_elems = v.row_elems;
                        r.pitch = v.pitch;
                        r.S = v.S;
                        int sl = v.slot0 + (s + ds - v.W0);
                        r.sl0 = sl >= v.S ? sl - v.S : sl;
                        return r;
                    };
                    d.orec = rec(d.v[0], 0, 0, 0);
                    for (int m = 0; m < ns; ++m)
                        d.srec[m] = rec(d.v[d.sarg[m]], d.soff[m][0], lp.ndim == 3 ? d.soff[m][1] : 0, d.soff[m][sa]);
                    d.lean = 1;
                    // 32-bit element offsets over every slab: the ring kernels address a
                    // row with one multiply-add (and a select only where a slab wraps)
                    auto fits = [&](const SampleRec& r) { return (long long)r.S * r.row_elems < (1LL << 31); };
                    bool ok = fits(d.orec);
                    for (int m = 0; m < ns && ok; ++m) ok = fits(d.srec[m]);
                    if (ok) {
                        d.ring = 1;
                        d.ore = (int)d.orec.row_elems;
                        for (int m = 0; m < ns; ++m) d.sre[m] = (int)d.srec[m].row_elems;
                    }
                }
            }
            // 32-bit element offsets inside every view (PDE kernels); uniform geometry:
            // one in-row offset per point serves every argument
            d.o32 = 1;
            d.uni = 1;
            int j0 = -1;
            for (int j = 0; j < d.nargs; ++j) {
                if (lp.args[j].access == OC_REDUCE) continue;
                const DView& v = d.v[j];
                if ((long long)v.S * v.row_elems >= (1LL << 31)) d.o32 = 0;
                if (j0 < 0) { j0 = j; continue; }
                const DView& w = d.v[j0];
                if (v.nx != w.nx || v.ny != w.ny || v.periodic != w.periodic || v.pitch != w.pitch ||
                    v.ox != w.ox || v.oy != w.oy)
                    d.uni = 0;
            }
            if (j0 != 0 || !d.o32) d.uni = 0;
            d.params = (const double*)(g->arena + sb + P.params_off) + P.loop_param[i];
            d.paramsf = (const float*)(g->arena + sb + P.paramsf_off) + P.loop_param[i];
            d.nparams = (int)lp.params.size();
            if (P.loop_red[i] >= 0) {
                d.part = (double*)(g->arena + sb + P.loop_part[i]);
                d.part_row0 = std::min(lp.lo[sa], lp.hi[sa]);
                d.chunks = P.loop_chunks[i];
                d.red_op = P.rp[P.loop_red[i]].op;
            }
            if (d.dtype < 0) d.dtype = OC_F64;
            out[t].push_back(d);
        }
}

static double launch_bytes(const LaunchDesc& d, double& points)
{
    points = 1;
    for (int a = 0; a < d.ndim; ++a) points *= (double)std::max(0, d.hi[a] - d.lo[a]);
    double b = 0;
    const double esz = d.dtype == OC_F32 ? 4 : 8;
    for (int j = 0; j < d.nargs; ++j)
        if (d.access[j] != OC_REDUCE) b += points * esz * (d.access[j] == OC_RW ? 2 : 1);
    return b;
}

static int pool_event(cudaEvent_t& ev, bool persistent)
{
    if (!persistent && g->ev_next < g->ev_pool.size()) { ev = g->ev_pool[g->ev_next++]; return OC_OK; }
    OC_CUDA(cudaEventCreate(&ev));
    if (!persistent) { g->ev_pool.push_back(ev); g->ev_next = g->ev_pool.size(); }
    return OC_OK;
}

// Launch the kernels of one tile on two compute streams: a loop that shares no dataset
// with a conflicting access (write/read, read/write, write/write) with its predecessor
// goes to the other stream, so that independent loops overlap and fill each other's
// last wave; every conflict with a loop on the other stream becomes an event wait.
// Program order is kept for every pair of loops that touch a common dataset, so the
// results are those of the serial order.
static int run_tile_two_streams(const std::vector<LaunchDesc>& ds, cudaStream_t s)
{
    const size_t n = ds.size();
    while (g->ev_launch.size() < n) {
        cudaEvent_t e;
        OC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        g->ev_launch.push_back(e);
    }
    // read / write sets of every launch, keyed by the dataset's device base address
    auto conflict = [&](const LaunchDesc& a, const LaunchDesc& b) {
        for (int i = 0; i < a.nargs; ++i) {
            if (a.access[i] == OC_REDUCE) continue;
            const bool aw = a.access[i] != OC_READ;
            for (int j = 0; j < b.nargs; ++j) {
                if (b.access[j] == OC_REDUCE || a.v[i].base != b.v[j].base) continue;
                if (aw || b.access[j] != OC_READ) return true;
            }
        }
        return false;
    };
    cudaStream_t st2[2] = {s, g->s0b};
    OC_CUDA(cudaEventRecord(g->ev_tf, s));
    OC_CUDA(cudaStreamWaitEvent(g->s0b, g->ev_tf, 0));
    std::vector<int> on(n, 0);
    bool used_b = false;
    for (size_t k = 0; k < n; ++k) {
        int last[2] = {-1, -1};   // latest conflicting launch on each stream
        for (size_t i = 0; i < k; ++i)
            if (conflict(ds[i], ds[k])) last[on[i]] = (int)i;
        int sk;
        if (k == 0) sk = 0;
        else if (last[0] < 0 && last[1] < 0) sk = 1 - on[k - 1];        // independent: alternate
        else sk = last[0] >= last[1] ? 0 : 1;                             // follow the latest conflict
        const int other = 1 - sk;
        if (last[other] >= 0) OC_CUDA(cudaStreamWaitEvent(st2[sk], g->ev_launch[last[other]], 0));
        on[k] = sk;
        used_b = used_b || sk == 1;
        int rc = OC_OK;
        if (injected(2)) rc = fail(OC_ERR_CUDA, "injected fault: launch of kernel %d", ds[k].kernel);
        cudaError_t e = rc ? cudaSuccess : launch_loop(ds[k], st2[sk]);
        if (e != cudaSuccess) rc = fail(OC_ERR_CUDA, "kernel %d launch failed: %s", ds[k].kernel, cudaGetErrorString(e));
        if (rc) {
            // join the second stream before giving up (a capture in progress can then end)
            cudaEventRecord(g->ev_tj, g->s0b);
            cudaStreamWaitEvent(s, g->ev_tj, 0);
            return rc;
        }
        OC_CUDA(cudaEventRecord(g->ev_launch[k], st2[sk]));
    }
    // join: everything after the tile on stream s sees both streams' work
    OC_CUDA(cudaEventRecord(g->ev_tj, g->s0b));
    OC_CUDA(cudaStreamWaitEvent(s, g->ev_tj, 0));
    (void)used_b;
    return OC_OK;
}

// Launch the kernels of one tile; with profiling, bracket each with events. `recs`
// receives the records (persistent events when the launches are being captured).
static int run_tile_kernels(const std::vector<LaunchDesc>& ds, cudaStream_t s,
                            std::vector<ProfRec>* recs = nullptr, bool persistent = false)
{
    // With OC_FLAG_PROFILE, each run of consecutive launches of one kernel id is
    // bracketed by one pair of events (an event between every two launches would
    // stall the launch pipeline and add its own gap to every launch).
    const bool prof = (g->flags & OC_FLAG_PROFILE) != 0 && !g->trial;
    if (!prof && !(g->flags & OC_FLAG_TRACE) && g->s0b && ds.size() > 1) return run_tile_two_streams(ds, s);
    const unsigned ext = persistent ? cudaEventRecordExternal : cudaEventRecordDefault;
    for (size_t k = 0; k < ds.size();) {
        size_t k1 = k + 1;
        if (prof)
            while (k1 < ds.size() && ds[k1].kernel == ds[k].kernel) ++k1;
        ProfRec pr{};
        if (prof) {
            int r = pool_event(pr.a, persistent);
            if (!r) r = pool_event(pr.b, persistent);
            if (r) return r;
            pr.kernel = ds[k].kernel;
            pr.launches = (int)(k1 - k);
            for (size_t j = k; j < k1; ++j) {
                double pts = 0;
                pr.bytes += launch_bytes(ds[j], pts);
                pr.points += pts;
            }
            // inside a stream capture only an "external" record becomes a graph node
            OC_CUDA(cudaEventRecordWithFlags(pr.a, s, ext));
        }
        for (size_t j = k; j < k1; ++j) {
            if (injected(2)) return fail(OC_ERR_CUDA, "injected fault: launch of kernel %d", ds[j].kernel);
            cudaError_t e = launch_loop(ds[j], s);
            if (e != cudaSuccess) return fail(OC_ERR_CUDA, "kernel %d launch failed: %s", ds[j].kernel, cudaGetErrorString(e));
        }
        if (prof) {
            OC_CUDA(cudaEventRecordWithFlags(pr.b, s, ext));
            if (recs) recs->push_back(pr);
            else g->prof_pending.push_back(pr);
        }
        k = k1;
    }
    return OC_OK;
}

static int trace_event(cudaEvent_t& ev)
{
    if (g->tr_next < g->tr_pool.size()) { ev = g->tr_pool[g->tr_next++]; return OC_OK; }
    OC_CUDA(cudaEventCreate(&ev));
    g->tr_pool.push_back(ev);
    g->tr_next = g->tr_pool.size();
    return OC_OK;
}

// Open / close one traced span on stream s (no-ops without OC_FLAG_TRACE).
static int trace_begin(int tile, int kind, cudaStream_t s)
{
    if (!(g->flags & OC_FLAG_TRACE) || g->trial) return OC_OK;
    Ctx::TraceRec r{tile, kind, nullptr, nullptr, 0.0};
    int rc = trace_event(r.a);
    if (!rc) rc = trace_event(r.b);
    if (rc) return rc;
    OC_CUDA(cudaEventRecord(r.a, s));
    g->tr.push_back(r);
    return OC_OK;
}

static int trace_end(cudaStream_t s, double bytes)
{
    if (!(g->flags & OC_FLAG_TRACE) || g->trial) return OC_OK;
    g->tr.back().bytes = bytes;
    OC_CUDA(cudaEventRecord(g->tr.back().b, s));
    return OC_OK;
}

static int collect_trace()
{
    g->tr_out.clear();
    for (const auto& r : g->tr) {
        float a = 0, b = 0;
        OC_CUDA(cudaEventElapsedTime(&a, g->tr_t0, r.a));
        OC_CUDA(cudaEventElapsedTime(&b, g->tr_t0, r.b));
        g->tr_out.push_back({r.tile, r.kind, (double)a, (double)b, r.bytes});
    }
    g->tr.clear();
    g->tr_next = 0;
    return OC_OK;
}

// After a chain has completed: fold the profiled launches into the per-kernel totals.
static int collect_profile()
{
    for (const ProfRec& pr : g->prof_pending) {
        float ms = 0;
        OC_CUDA(cudaEventElapsedTime(&ms, pr.a, pr.b));
        KStat& k = g->kstats[pr.kernel];
        k.launches += pr.launches;
        k.ms += ms;
        k.bytes += pr.bytes;
        k.points += pr.points;
    }
    g->prof_pending.clear();
    g->ev_next = 0;
    return OC_OK;
}

static int count_launches(const std::vector<LaunchDesc>& ds) { return (int)ds.size(); }

// ---------------------------------------------------------------------------------
static long long resident_total()
{
    long long tot = 0;
    for (const Dat& d : g->dats) tot += align_up(d.bytes(), 256);
    return tot;
}

static int leave_resident_mode()
{
    for (Dat& d : g->dats) {
        if (d.resident && !d.host_valid && d.dev_valid && !g->dryrun) {
            OC_CUDA(cudaMemcpyAsync(d.host, g->arena + d.res_off, (size_t)d.bytes(),
                                    cudaMemcpyDeviceToHost, g->st[2]));
        }
    }
    if (!g->dryrun) { int r = wait_stream(g->st[2]); if (r) return r; }
    for (Dat& d : g->dats) { d.resident = false; d.dev_valid = false; d.host_valid = true; d.res_off = -1; }
    g->resident_mode = false;
    return OC_OK;
}

static void enter_resident_layout()
{
    long long off = 0;
    for (Dat& d : g->dats) {
        if (!d.resident) { d.resident = true; d.dev_valid = false; }
        d.res_off = off;
        off += align_up(d.bytes(), 256);
    }
    g->resident_bytes = off;
    g->resident_mode = true;
}

// Partial residency (streamed plans that keep some datasets whole in the arena). A
// dataset resident now but not kept by `keep` at the same offset goes home first: its
// device copy is downloaded if the host copy is stale, then it is streamed again (or
// placed anew). keep == nullptr releases every partially resident dataset.
static int release_residents(const Plan* keep)
{
    if (g->resident_mode || g->dryrun) return OC_OK;
    std::vector<int> drop;
    for (size_t k = 0; k < g->dats.size(); ++k) {
        Dat& d = g->dats[k];
        if (!d.resident) continue;
        bool kept = false;
        if (keep && k < keep->dat_index.size() && keep->dat_index[k] >= 0) {
            const DatPlan& dp = keep->dp[keep->dat_index[k]];
            kept = dp.resident && dp.off == d.res_off;
        }
        if (kept) continue;
        if (d.dev_valid && !d.host_valid)
            OC_CUDA(cudaMemcpyAsync(d.host, g->arena + d.res_off, (size_t)d.bytes(), cudaMemcpyDeviceToHost, g->st[2]));
        drop.push_back((int)k);
    }
    if (drop.empty()) return OC_OK;
    int r = wait_stream(g->st[2]);
    if (r) return r;
    for (int k : drop) {
        Dat& d = g->dats[k];
        d.resident = false;
        d.dev_valid = false;
        d.host_valid = true;
        d.res_off = -1;
    }
    return OC_OK;
}

// Make the datasets plan P keeps resident resident at their offsets (their upload
// happens with the chain, on the upload stream, while the device copy is not current).
static int apply_residency(const Plan& P)
{
    int r = release_residents(&P);
    if (r) return r;
    for (const DatPlan& dp : P.dp) {
        if (!dp.resident) continue;
        Dat& d = g->dats[dp.dat];
        if (!d.resident) {
            d.resident = true;
            d.res_off = dp.off;
            d.dev_valid = false;
        }
    }
    return OC_OK;
}

static bool residents_pending(const Plan& P)
{
    for (const DatPlan& dp : P.dp)
        if (dp.resident && !g->dats[dp.dat].dev_valid) return true;
    return false;
}

// Refresh the halo rows of a periodic slow axis from the opposite end (deep ghosts).
// Deep ghost rows of a periodic slow axis on the host: row y < 0 or y >= n takes the
// interior row y mod n. The rows are copied on several threads when there are tens of
// MB of them (3-D datasets), since the chain waits for them.
static int ghost_fill_host(const Dat& d)
{
    const int sa = d.slow();
    const int n = d.size[sa], lo = d.hlo[sa], hi = d.hhi[sa];
    const long long rb = d.row_bytes();
    char* h = (char*)d.host;
    auto row = [&](int y) { return h + (long long)(y - d.y0) * rb; };
    const int ng = lo + hi;
    if (-lo < d.y0 || n + hi > d.y0 + d.nrows)
        return fail(OC_ERR_STATE, "periodic ghost rows [%d, %d) outside the host store's rows [%d, %d)",
                    -lo, n + hi, d.y0, d.y0 + d.nrows);
    auto fill = [&](int k0, int k1) {
        for (int k = k0; k < k1; ++k) {
            const int y = k < lo ? k - lo : n + (k - lo);
            const int src = ((y % n) + n) % n;
            memcpy(row(y), row(src), (size_t)rb);
        }
    };
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nt = (int)std::min<long long>(std::min<unsigned>(hw, 8), (long long)ng * rb / (4LL << 20));
    if (nt <= 1) {
        fill(0, ng);
        return OC_OK;
    }
    std::vector<std::thread> th;
    const int per = (ng + nt - 1) / nt;
    for (int t = 1; t < nt; ++t) {
        const int k0 = t * per, k1 = std::min(ng, k0 + per);
        if (k0 < k1) th.emplace_back(fill, k0, k1);
    }
    fill(0, std::min(ng, per));
    for (auto& t : th) t.join();
    return OC_OK;
}

// Deep ghost rows of a dataset held whole in the arena at byte offset `off` (in-core or
// resident), refreshed on the device.
static int ghost_fill_device(const Dat& d, long long off, cudaStream_t s)
{
    const int sa = d.slow();
    const int n = d.size[sa], lo = d.hlo[sa], hi = d.hhi[sa];
    const long long rb = d.row_bytes();
    if (off < 0 || off + d.bytes() > g->arena_bytes)
        return fail(OC_ERR_STATE, "ghost refresh of dataset outside the arena (offset %lld)", off);
    char* b = g->arena + off;
    auto row = [&](int y) { return b + (long long)(y + lo) * rb; };
    // ghost row y takes interior row y mod n: runs of consecutive rows, one copy each
    auto fill = [&](int y, int end) -> int {
        while (y < end) {
            const int src = ((y % n) + n) % n;
            const int len = std::min(end - y, n - src);
            OC_CUDA(cudaMemcpyAsync(row(y), row(src), (size_t)len * rb, cudaMemcpyDeviceToDevice, s));
            y += len;
        }
        return OC_OK;
    };
    int rc = fill(-lo, 0);
    if (!rc) rc = fill(n, n + hi);
    return rc;
}

// True if the chain reads a ghost row of the dataset before writing it (the row is
// uploaded, whole or in columns): only then does the ghost copy have to be refreshed.
// Ghost rows the chain computes first (temporaries extended into the ghosts) need none.
static bool reads_ghosts(const Plan& P, int di)
{
    const DatPlan& dp = P.dp[di];
    const Dat& d = g->dats[dp.dat];
    const int sa = d.slow();
    for (int r = 0; r < dp.nrows; ++r) {
        int y = r + dp.y0;
        if ((y < 0 || y >= d.size[sa]) && dp.first[r] >= 0 && dp.need_up[r]) return true;
    }
    return false;
}

// ---------------------------------------------------------------------------------
static int run_plan(Plan& P, const std::vector<Loop>& loops, bool trial, double* ms_out,
                    std::chrono::steady_clock::time_point t0);

// Exhaustive autotuner (OC_PLAN_AUTOTUNE): every candidate of the grid -- residency level
// (kResLevel), depth 2..4 and kGridN tile heights (fractions of the largest that fits at
// that depth and residency) -- runs the chain as a side-effect-free trial, in
// kTuneRounds interleaved rounds; a candidate's time is the median of its rounds and the
// fastest candidate wins. Partially resident datasets are released first, so that trials
// find every host copy current.
constexpr int kTuneRounds = 3;

static int autotune(const std::vector<Loop>& loops, PlanChoice& best_c, int& h_best)
{
    std::string err;
    int rc = release_residents(nullptr);
    if (rc) return rc;
    g->tune.clear();
    struct Cand { PlanChoice c; int h, hmax; Plan P; std::vector<double> ms; };
    std::vector<Cand> cands;
    std::vector<long long> prev_off;
    for (int ri = 0; ri < kResN; ++ri) {
        if (g->force_res >= 0 && ri > 0) break;
        const Residency R = choose_residency(loops, g->dats, g->red_ops, g->flags, g->budget,
                                             g->force_res >= 0 ? g->force_res : kResLevel[ri]);
        if (ri > 0 && (!R.any() || R.off == prev_off)) continue;   // nothing new at this level
        prev_off = R.off;
        for (int depth = 2; depth <= 4; ++depth) {
            const int hmax = fit_tile_height(loops, g->dats, g->red_ops, depth, g->flags, g->budget, err, &R);
            if (hmax <= 0) continue;
            int prev = -1;
            for (int gi = 0; gi < kGridN; ++gi) {
                const int h = grid_height(hmax, gi);
                if (h == prev) continue;
                prev = h;
                Cand c;
                c.c = PlanChoice{gi, depth, ri};
                c.h = h;
                c.hmax = hmax;
                build_plan(loops, g->dats, g->red_ops, h, depth, g->flags, false, c.P, err, &R);
                if (c.P.arena_bytes > g->budget) continue;
                cands.push_back(std::move(c));
            }
        }
    }
    for (int round = 0; round < kTuneRounds; ++round)
        for (Cand& c : cands) {
            double m = 0;
            rc = run_plan(c.P, loops, true, &m, std::chrono::steady_clock::now());
            g->trial = false;
            if (rc) return rc;
            c.ms.push_back(m);
        }
    double best = 1e300;
    h_best = 0;
    for (Cand& c : cands) {
        g->descs.erase(c.P.sig);
        std::sort(c.ms.begin(), c.ms.end());
        const double ms = c.ms[c.ms.size() / 2];
        g->tune.push_back({(double)c.h, (double)c.c.depth, ms, (double)c.c.grid, (double)c.hmax,
                           g->force_res >= 0 ? g->force_res : kResLevel[c.c.res]});
        if (ms < best) { best = ms; h_best = c.h; best_c = c.c; }
    }
    return OC_OK;
}

static int select_plan_uncached(const std::vector<Loop>& loops, uint64_t csig, Plan*& out)
{
    std::string err;
    // in-core (resident) mode when every declared dataset fits with the scratch
    Plan inc;
    build_plan(loops, g->dats, g->red_ops, 0, 3, g->flags, true, inc, err);
    const long long rtot = resident_total();
    const bool managed = (g->flags & OC_FLAG_MANAGED) != 0;
    if (!managed && rtot + inc.scratch_bytes <= g->budget && g->force_h == 0) {
        if (!g->resident_mode) {
            int r = release_residents(nullptr);
            if (r) return r;
            enter_resident_layout();
        } else {  // new datasets since the layout was made
            long long off = 0;
            for (Dat& d : g->dats) {
                if (!d.resident) { d.resident = true; d.dev_valid = false; d.res_off = off; }
                off = std::max(off, d.res_off + align_up(d.bytes(), 256));
            }
            g->resident_bytes = off;
        }
        uint64_t key = inc.sig ^ 0x1234567ull ^ ((uint64_t)g->resident_bytes * 0x9E3779B97F4A7C15ull);
        auto it = g->plans.find(key);
        if (it == g->plans.end()) { inc.sig = key; it = g->plans.emplace(key, std::move(inc)).first; }
        out = &it->second;
        return OC_OK;
    }
    if (g->resident_mode) { int r = leave_resident_mode(); if (r) return r; }

    int h = 0;
    PlanChoice choice = kFixedChoice;
    if (g->force_depth > 0) choice.depth = g->force_depth;
    chain_features(loops, g->dats, g->budget, g->features);
    if (g->force_h <= 0 && g->force_depth <= 0 && g->planner_mode != OC_PLAN_FIXED && !g->dryrun && !managed) {
        if (!(g->planner_mode == OC_PLAN_LEARNED && g->force_res < 0 && planner_predict(g->features, choice))) {
            int rc = autotune(loops, choice, h);
            if (rc) return rc;
        }
    }
    const double level = managed ? 0.0 : (g->force_res >= 0 ? g->force_res : kResLevel[choice.res]);
    const Residency R = choose_residency(loops, g->dats, g->red_ops, g->flags, g->budget, level);
    const int depth = choice.depth;
    if (h <= 0) {
        if (g->force_h > 0) h = g->force_h;
        else {
            const int hmax = fit_tile_height(loops, g->dats, g->red_ops, depth, g->flags, g->budget, err, &R);
            h = hmax > 0 ? grid_height(hmax, choice.grid) : 0;
        }
    }
    if (h <= 0) return fail(OC_ERR_BUDGET, "device budget of %lld bytes cannot hold one tile of height 1", g->budget);
    Plan P;
    build_plan(loops, g->dats, g->red_ops, h, depth, g->flags, false, P, err, &R);
    if (P.arena_bytes > g->budget)
        return fail(OC_ERR_BUDGET, "plan with tile height %d depth %d needs %lld bytes > budget %lld", h,
                    depth, P.arena_bytes, g->budget);
    auto it = g->plans.find(P.sig);
    if (it == g->plans.end()) it = g->plans.emplace(P.sig, std::move(P)).first;
    out = &it->second;
    (void)csig;
    return OC_OK;
}

// Plan of a chain: the choice (in-core or streamed, tile height, depth) is made once per
// chain shape, tiling override, planner mode and number of declared datasets.
static int select_plan(const std::vector<Loop>& loops, Plan*& out)
{
    uint64_t key = chain_signature(loops, g->dats, g->flags);
    key ^= ((uint64_t)(uint32_t)g->force_h << 20) ^ ((uint64_t)g->force_depth << 52) ^
           ((uint64_t)g->planner_mode << 60) ^ ((uint64_t)g->dats.size() * 0xC2B2AE3D27D4EB4Full) ^
           ((uint64_t)(int64_t)std::llround(g->force_res * 1e6) * 0x165667B19E3779F9ull);
    auto it = g->chosen.find(key);
    if (it != g->chosen.end() && (!it->second->incore || g->resident_mode)) {
        out = it->second;
        return OC_OK;
    }
    int rc = select_plan_uncached(loops, key, out);
    if (rc) return rc;
    g->chosen[key] = out;
    return OC_OK;
}

// Unified Memory variant (OC_FLAG_MANAGED, Sec. 5.4): the rows of dataset d whose first
// (to_gpu) or last tile is t, in runs of consecutive rows, are prefetched to the GPU or
// back to the host on stream s. A tile's device-bound prefetches take the place of its
// uploads, its host-bound ones of its downloads.
static int managed_prefetch(const DatPlan& dp, const Dat& d, int t, bool to_gpu, cudaStream_t s, double& bytes)
{
    const std::vector<int>& tile = to_gpu ? dp.first : dp.last;
    cudaMemLocation loc;
    loc.type = to_gpu ? cudaMemLocationTypeDevice : cudaMemLocationTypeHost;
    loc.id = 0;
    if (to_gpu) OC_CUDA(cudaGetDevice(&loc.id));
    const long long rb = d.row_bytes();
    int r = 0;
    while (r < dp.nrows) {
        if (dp.first[r] < 0 || tile[r] != t) { ++r; continue; }
        const int a = r;
        while (r < dp.nrows && dp.first[r] >= 0 && tile[r] == t) ++r;
        if (injected(to_gpu ? 0 : 1))
            return fail(OC_ERR_CUDA, "injected fault: %s prefetch of rows [%d, %d)", to_gpu ? "device" : "host",
                        a + dp.y0, r + dp.y0);
        OC_CUDA(cudaMemPrefetchAsync((char*)d.host + (long long)a * rb, (size_t)(r - a) * rb, loc, 0, s));
        bytes += (double)(r - a) * rb;
    }
    return OC_OK;
}

// Prefetch the first tile of a chain assumed to repeat this plan (Sec. 4.1). Only
// rows whose slots are not live in the last two phases (T - 1 and T) are fetched, so
// the prefetch starts as soon as phase T - 2 is done -- in phase T - 1, where the
// upload stream has nothing else to move -- and only rows whose host copy is final by
// then (not downloaded in phases T - 1 or T); ghost rows of a periodic slow axis are
// left out (they are refreshed when the next chain starts).
static int issue_prefetch(const Plan& P)
{
    g->pf.active = false;
    g->pf.rows.assign(P.dp.size(), {});
    g->pf.bytes = 0;
    if (P.T < 2 || P.incore) return OC_OK;
    const int T = P.T;
    StripBatch strips;
    strips.njobs = 0;
    OC_CUDA(cudaStreamWaitEvent(g->st[1], g->ev_comp[T - 2], 0));
    if (T >= 3 && g->dn_rec[T - 3]) OC_CUDA(cudaStreamWaitEvent(g->st[1], g->ev_down[T - 3], 0));
    bool any = false;
    for (size_t di = 0; di < P.dp.size(); ++di) {
        const DatPlan& dp = P.dp[di];
        const Dat& d = g->dats[dp.dat];
        const int sa = d.slow();
        // slots live in phases T-1 and T
        std::vector<uint8_t> busy(dp.S, 0);
        for (int r = 0; r < dp.nrows; ++r) {
            if (dp.first[r] < 0) continue;
            int pe = dp.dl[r] ? dp.last[r] + 1 : dp.last[r];
            if (pe >= T - 1) busy[r % dp.S] = 1;
        }
        bool ok = true;
        std::vector<Interval> rows;
        for (const Interval& iv : dp.up) {
            if (iv.t != 0) continue;
            for (int y = iv.a; y < iv.b; ++y) {
                int r = y - dp.y0;
                bool ghost = (d.periodic & (1 << sa)) && (y < 0 || y >= d.size[sa]);
                if (ghost) continue;
                if (busy[r % dp.S] || (dp.dl[r] && dp.last[r] >= T - 2)) { ok = false; break; }
                if (!rows.empty() && rows.back().b == y && rows.back().x0 == iv.x0 && rows.back().x1 == iv.x1)
                    rows.back().b = y + 1;
                else rows.push_back({0, y, y + 1, iv.x0, iv.x1});
            }
            if (!ok) break;
        }
        if (!ok) continue;
        for (const Interval& iv : rows) {
            double b = 0;
            int r = copy_rows(d, g->arena + dp.off, dp.S, iv.a, iv.b, true, g->st[1], b, iv.x0, iv.x1, nullptr,
                              &strips, &g->stats);
            if (r) return r;
            g->pf.bytes += b;
        }
        g->pf.rows[di] = rows;
        any = any || !rows.empty();
    }
    int rs = flush_strips(strips, g->st[1], &g->stats);
    if (rs) return rs;
    if (!any) return OC_OK;   // nothing fetched: no event for the next chain to wait on
    OC_CUDA(cudaEventRecord(g->ev_pf, g->st[1]));
    g->pf.active = true;
    g->pf.sig = P.sig;
    return OC_OK;
}

static int issue_chain(Plan& P, const std::vector<Loop>& loops, bool trial, bool capturing, bool pf_match,
                       oc_stats_t& S, long long sb, const double* hp, const float* hpf, double* hr);
static int finish_chain(Plan& P, const std::vector<Loop>& loops, bool trial, bool graphed, double* ms_out,
                        oc_stats_t& S, std::chrono::steady_clock::time_point t0, const double* hr);

// Run one chain with plan P. In a trial (autotuning) nothing the user can observe
// changes: downloads land in a scratch buffer, reduction results are dropped, no
// prefetch, graphs, trace or profile; *ms_out receives the device time of the chain.
static int run_plan(Plan& P, const std::vector<Loop>& loops, bool trial, double* ms_out,
                    std::chrono::steady_clock::time_point t0)
{
    oc_stats_t dummy{};
    oc_stats_t& S = trial ? dummy : g->stats;
    g->trial = trial;
    if (trial) {
        size_t need = 1;
        for (const DatPlan& dp : P.dp)
            if (!dp.resident) need = std::max(need, (size_t)dp.S * (size_t)g->dats[dp.dat].row_bytes());
        if (need > g->trial_sink_bytes) {
            host_free(g->trial_sink, true);
            g->trial_sink = (char*)host_alloc(need, true);
            if (!g->trial_sink) { g->trial_sink_bytes = 0; return fail(OC_ERR_NOMEM, "pinned trial buffer"); }
            g->trial_sink_bytes = need;
        }
    }
    auto dit = g->descs.find(P.sig);
    if (dit == g->descs.end()) {
        dit = g->descs.emplace(P.sig, std::vector<std::vector<LaunchDesc>>()).first;
        build_descs(P, loops, dit->second);
    }
    (void)dit;
    cudaStream_t s0 = g->st[0], s1 = g->st[1], s2 = g->st[2];
    int rc = ensure_events(std::max(P.T, 1));
    if (rc) return rc;
    if (!trial && !P.incore) {
        rc = apply_residency(P);
        if (rc) return rc;
    }

    // parameters of every loop, one block
    if ((size_t)P.nparams > g->h_params_cap) {
        host_free(g->h_params, true);
        g->h_params_cap = std::max<size_t>(P.nparams, 1024);
        g->h_params = (double*)host_alloc(g->h_params_cap * 12, true);
        if (!g->h_params) return fail(OC_ERR_NOMEM, "pinned parameter block");
    }
    float* h_paramsf = (float*)(g->h_params + g->h_params_cap);
    if (g->h_results_cap < P.rp.size() || !g->h_results) {
        host_free(g->h_results, true);
        g->h_results_cap = std::max<size_t>(P.rp.size(), 64);
        g->h_results = (double*)host_alloc(g->h_results_cap * 8, true);
        if (!g->h_results) return fail(OC_ERR_NOMEM, "pinned result block");
    }
    for (int i = 0; i < P.L; ++i)
        for (size_t j = 0; j < loops[i].params.size(); ++j) {
            g->h_params[P.loop_param[i] + j] = loops[i].params[j];
            h_paramsf[P.loop_param[i] + j] = (float)loops[i].params[j];
        }
    const long long sb = scratch_base(P);

    // a prefetch made for another plan (or before a trial) must land before anything
    // else touches slots
    bool pf_match = !trial && g->pf.active && g->pf.sig == P.sig && !P.incore;
    if (g->pf.active) {
        for (int k = 0; k < 3; ++k) OC_CUDA(cudaStreamWaitEvent(g->st[k], g->ev_pf, 0));
        if (!pf_match) g->pf.active = false;
    }
    if (trial) {
        // a trial measures the steady state of a plan: its resident datasets go up before
        // the timing starts (from the host store, which trials never change)
        bool up = false;
        for (const DatPlan& dp : P.dp) {
            if (!dp.resident) continue;
            const Dat& d = g->dats[dp.dat];
            OC_CUDA(cudaMemcpyAsync(g->arena + dp.off, d.host, (size_t)d.bytes(), cudaMemcpyHostToDevice, s1));
            up = true;
        }
        if (up) {
            OC_CUDA(cudaEventRecord(g->ev_resup, s1));
            OC_CUDA(cudaStreamWaitEvent(s0, g->ev_resup, 0));
        }
        OC_CUDA(cudaEventRecord(g->tm0, s0));
        OC_CUDA(cudaStreamWaitEvent(s1, g->tm0, 0));
        OC_CUDA(cudaStreamWaitEvent(s2, g->tm0, 0));
    }

    if (!trial && (g->flags & OC_FLAG_TRACE)) {
        if (!g->tr_t0) OC_CUDA(cudaEventCreate(&g->tr_t0));
        OC_CUDA(cudaEventRecord(g->tr_t0, s0));
        OC_CUDA(cudaStreamWaitEvent(s1, g->tr_t0, 0));
        OC_CUDA(cudaStreamWaitEvent(s2, g->tr_t0, 0));
        g->tr.clear();
        g->tr_next = 0;
    }
    // the chain's upload and download streams start after all earlier work of stream 0
    // (the previous chain's whole-chain graph included)
    OC_CUDA(cudaEventRecord(g->ev_fork, s0));
    OC_CUDA(cudaStreamWaitEvent(s1, g->ev_fork, 0));
    OC_CUDA(cudaStreamWaitEvent(s2, g->ev_fork, 0));
    bool incore_uploads = false;
    if (P.incore)
        for (const DatPlan& dp : P.dp) incore_uploads = incore_uploads || !g->dats[dp.dat].dev_valid;
    const bool chain_graph = !trial && (g->flags & OC_FLAG_GRAPHS) && !(g->flags & (OC_FLAG_TRACE | OC_FLAG_PROFILE)) &&
                             !incore_uploads && !(!P.incore && residents_pending(P)) &&
                             !(g->flags & OC_FLAG_MANAGED);
    ChainGraph* cg = nullptr;
    bool replay = false;
    if (chain_graph) {
        const uint64_t key = P.sig ^ (pf_match ? 0x9E3779B1ull : 0) ^ ((g->flags & OC_FLAG_PREFETCH) ? (0x7F4A7C15ull << 20) : 0);
        cg = &g->chain_graphs[key];
        replay = cg->exec != nullptr;
    }
    // staging of parameters and results: the context's buffers, or the graph's own (a
    // captured copy node keeps its host address for the graph's lifetime); pinned host
    // memory cannot be allocated while a stream is being captured
    const double* hp = g->h_params;
    const float* hpf = h_paramsf;
    double* hr = g->h_results;
    if (chain_graph) {
        if (!cg->hp) {
            cg->hp = (double*)host_alloc((size_t)std::max(1, P.nparams) * 12, true);
            cg->hr = (double*)host_alloc(std::max<size_t>(1, P.rp.size()) * 8, true);
            if (!cg->hp || !cg->hr) return fail(OC_ERR_NOMEM, "pinned graph staging");
        }
        memcpy(cg->hp, g->h_params, (size_t)P.nparams * 8);
        memcpy(cg->hp + std::max(1, P.nparams), h_paramsf, (size_t)P.nparams * 4);
        hp = cg->hp;
        hpf = (const float*)(cg->hp + std::max(1, P.nparams));
        hr = cg->hr;
        if (!replay) {
            OC_CUDA(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
            cudaError_t e1 = cudaEventRecord(g->ev_fork2, s0);
            cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(s1, g->ev_fork2, 0) : e1;
            cudaError_t e3 = e2 == cudaSuccess ? cudaStreamWaitEvent(s2, g->ev_fork2, 0) : e2;
            if (e3 != cudaSuccess) {
                cudaGraph_t tmp;
                cudaStreamEndCapture(s0, &tmp);
                if (tmp) cudaGraphDestroy(tmp);
                return fail(OC_ERR_CUDA, "chain capture failed: %s", cudaGetErrorString(e3));
            }
        }
    }
    if (!replay) {
        rc = issue_chain(P, loops, trial, chain_graph, pf_match, S, sb, hp, hpf, hr);
        if (chain_graph) {
            // the copy streams join the compute stream even after a failure, so that the
            // capture ends cleanly and no stream is left in capture mode
            cudaError_t e = cudaEventRecord(g->ev_j1, s1);
            if (e == cudaSuccess) e = cudaEventRecord(g->ev_j2, s2);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s0, g->ev_j1, 0);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s0, g->ev_j2, 0);
            cudaGraph_t gr = nullptr;
            cudaError_t ce = cudaStreamEndCapture(s0, &gr);
            if (rc || e != cudaSuccess || ce != cudaSuccess) {
                if (gr) cudaGraphDestroy(gr);
                if (rc) return rc;
                return fail(OC_ERR_CUDA, "chain capture failed: %s",
                            cudaGetErrorString(e != cudaSuccess ? e : ce));
            }
            cudaError_t ie = cudaGraphInstantiate(&cg->exec, gr, 0);
            cudaGraphDestroy(gr);
            if (ie != cudaSuccess) return fail(OC_ERR_CUDA, "chain graph instantiation failed: %s", cudaGetErrorString(ie));
            cg->h2d = S.h2d_bytes;
            cg->d2h = S.d2h_bytes;
            cg->prefetched = S.prefetched_bytes;
            cg->launches = S.kernel_launches;
            cg->pf_active = g->pf.active;
            cg->pf_sig = g->pf.sig;
            cg->pf_bytes = g->pf.bytes;
            cg->pf_rows = g->pf.rows;
        } else if (rc) {
            return rc;
        }
    } else {
        S.h2d_bytes = cg->h2d;
        S.d2h_bytes = cg->d2h;
        S.prefetched_bytes = cg->prefetched;
        S.kernel_launches = cg->launches;
        S.graph_replays = P.T;
        g->pf.active = cg->pf_active;
        g->pf.sig = cg->pf_sig;
        g->pf.bytes = cg->pf_bytes;
        g->pf.rows = cg->pf_rows;
        if (!P.incore)
            for (size_t di = 0; di < P.dp.size(); ++di) {
                const Dat& d = g->dats[P.dp[di].dat];
                if (!P.dp[di].resident && (d.periodic & (1 << d.slow())) && reads_ghosts(P, (int)di)) {
                    const int r = ghost_fill_host(d);
                    if (r) return r;
                }
            }
        if (P.res_dats > 0)
            for (const Loop& lp : loops)
                for (const Arg& ar : lp.args)
                    if ((ar.access == OC_WRITE || ar.access == OC_RW) && P.dat_index[ar.dat] >= 0 &&
                        P.dp[P.dat_index[ar.dat]].resident)
                        g->dats[ar.dat].host_valid = false;
    }
    if (chain_graph) {
        OC_CUDA(cudaGraphLaunch(cg->exec, s0));
        // the prefetch event recorded inside the capture is a graph node; the next chain
        // waits on a real event, which the graph's end (it joins the copy streams) covers
        if (g->pf.active) OC_CUDA(cudaEventRecord(g->ev_pf, s0));
    }
    return finish_chain(P, loops, trial, chain_graph, ms_out, S, t0, hr);
}

// Issue every asynchronous operation of one chain on the three streams (optionally
// inside a stream capture: then no per-tile graphs, trace or profile).
static int issue_chain(Plan& P, const std::vector<Loop>& loops, bool trial, bool capturing, bool pf_match,
                       oc_stats_t& S, long long sb, const double* hp, const float* hpf, double* hr)
{
    cudaStream_t s0 = g->st[0], s1 = g->st[1], s2 = g->st[2];
    int rc = OC_OK;
    const auto& tdesc = g->descs[P.sig];
    // The compute stream carries no copy of its own: after a copy, a stream's next wait
    // was seen to be served behind the copy engine's queue, so that the first tile's
    // kernels started only once the next bulk upload had finished. The parameters go
    // first on the upload stream; the results come back on the download stream.
    if (P.nparams > 0) {
        OC_CUDA(cudaMemcpyAsync(g->arena + sb + P.params_off, hp, (size_t)P.nparams * 8,
                                cudaMemcpyHostToDevice, s1));
        OC_CUDA(cudaMemcpyAsync(g->arena + sb + P.paramsf_off, hpf, (size_t)P.nparams * 4,
                                cudaMemcpyHostToDevice, s1));
        OC_CUDA(cudaEventRecord(g->ev_par, s1));
        OC_CUDA(cudaStreamWaitEvent(s0, g->ev_par, 0));
    }

    const bool use_graphs = !trial && !capturing && (g->flags & OC_FLAG_GRAPHS) != 0;
    GraphSet* gs = nullptr;
    if (use_graphs) {
        gs = &g->graphs[P.sig ^ ((g->flags & OC_FLAG_PROFILE) ? 0xABCDEFull : 0)];
        if (gs->tiles.size() < (size_t)P.T) { gs->tiles.resize(P.T, nullptr); gs->prof.resize(P.T); }
    }
    auto run_compute = [&](int t) -> int {
        if (use_graphs) {
            if (!gs->tiles[t]) {
                cudaGraph_t gr;
                OC_CUDA(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
                int r = run_tile_kernels(tdesc[t], s0, &gs->prof[t], true);
                cudaError_t ce = cudaStreamEndCapture(s0, &gr);
                if (r) return r;
                if (ce != cudaSuccess) return fail(OC_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
                OC_CUDA(cudaGraphInstantiate(&gs->tiles[t], gr, 0));
                cudaGraphDestroy(gr);
            } else {
                S.graph_replays++;
            }
            OC_CUDA(cudaGraphLaunch(gs->tiles[t], s0));
            for (const ProfRec& pr : gs->prof[t]) g->prof_pending.push_back(pr);
        } else {
            int r = run_tile_kernels(tdesc[t], s0);
            if (r) return r;
        }
        S.kernel_launches += count_launches(tdesc[t]);
        return OC_OK;
    };

    if (P.incore) {
        // in-core: datasets stay resident; upload whatever is not on the device yet
        bool up = false;
        for (size_t di = 0; di < P.dp.size(); ++di) {
            Dat& d = g->dats[P.dp[di].dat];
            if (!d.dev_valid) {
                OC_CUDA(cudaMemcpyAsync(g->arena + d.res_off, d.host, (size_t)d.bytes(), cudaMemcpyHostToDevice, s1));
                S.h2d_bytes += (double)d.bytes();
                d.dev_valid = true;
                up = true;
            }
        }
        if (up) {
            OC_CUDA(cudaEventRecord(g->ev_up[0], s1));
            OC_CUDA(cudaStreamWaitEvent(s0, g->ev_up[0], 0));
        }
        for (size_t di = 0; di < P.dp.size(); ++di) {
            Dat& d = g->dats[P.dp[di].dat];
            if ((d.periodic & (1 << d.slow())) && reads_ghosts(P, (int)di)) {
                rc = ghost_fill_device(d, d.res_off, s0);
                if (rc) return rc;
            }
        }
        if (P.T > 0) {
            rc = trace_begin(0, 1, s0);
            if (!rc) rc = run_compute(0);
            if (!rc) rc = trace_end(s0, 0.0);
            if (rc) return rc;
        }
        if (!trial)
            for (const Loop& lp : loops)
                for (const Arg& ar : lp.args)
                    if (ar.access == OC_WRITE || ar.access == OC_RW) g->dats[ar.dat].host_valid = false;
    } else {
        for (size_t di = 0; di < P.dp.size(); ++di) {
            const Dat& d = g->dats[P.dp[di].dat];
            if (!P.dp[di].resident && (d.periodic & (1 << d.slow())) && reads_ghosts(P, (int)di)) {
                rc = ghost_fill_host(d);
                if (rc) return rc;
            }
        }
        // datasets the plan keeps resident: uploaded whole while their device copy is not
        // current (a trial uploaded them before its timing started), deep ghosts refreshed
        // on the device
        if (P.res_dats > 0) {
            bool up = false;
            for (const DatPlan& dp : P.dp) {
                if (!dp.resident) continue;
                Dat& d = g->dats[dp.dat];
                if (trial || d.dev_valid) continue;
                OC_CUDA(cudaMemcpyAsync(g->arena + dp.off, d.host, (size_t)d.bytes(), cudaMemcpyHostToDevice, s1));
                S.h2d_bytes += (double)d.bytes();
                d.dev_valid = true;
                up = true;
            }
            if (up) {
                OC_CUDA(cudaEventRecord(g->ev_resup, s1));
                OC_CUDA(cudaStreamWaitEvent(s0, g->ev_resup, 0));
            }
            for (size_t di = 0; di < P.dp.size(); ++di) {
                const Dat& d = g->dats[P.dp[di].dat];
                if (P.dp[di].resident && (d.periodic & (1 << d.slow())) && reads_ghosts(P, (int)di)) {
                    // the plan's offset: a trial runs without applying the residency
                    rc = ghost_fill_device(d, P.dp[di].off, s0);
                    if (rc) return rc;
                }
            }
            if (!trial)
                for (const Loop& lp : loops)
                    for (const Arg& ar : lp.args)
                        if ((ar.access == OC_WRITE || ar.access == OC_RW) && P.dat_index[ar.dat] >= 0 &&
                            P.dp[P.dat_index[ar.dat]].resident)
                            g->dats[ar.dat].host_valid = false;
        }
        const int T = P.T, k = P.depth - 2;
        g->up_rec.assign(std::max(T, 1), 0);
        g->dn_rec.assign(std::max(T, 1), 0);
        for (int p = -k; p <= T; ++p) {
            const int u = p + k;
            // Issue order inside a phase: with lookahead (k >= 1) compute and download
            // go first so the compute stream is fed before the host spends time on the
            // upload calls; with k == 0 the upload of tile p must be issued before the
            // compute that waits for it.
            if (k >= 1 && p >= 0 && p < T) {
                if (g->up_rec[p]) OC_CUDA(cudaStreamWaitEvent(s0, g->ev_up[p], 0));
                if (p - 2 >= 0 && g->dn_rec[p - 2]) OC_CUDA(cudaStreamWaitEvent(s0, g->ev_down[p - 2], 0));
                rc = trace_begin(p, 1, s0);
                if (!rc) rc = run_compute(p);
                if (!rc) rc = trace_end(s0, 0.0);
                if (rc) return rc;
                OC_CUDA(cudaEventRecord(g->ev_comp[p], s0));
            }
            if (u >= 0 && u < T) {
                if (p - 1 >= 0) OC_CUDA(cudaStreamWaitEvent(s1, g->ev_comp[p - 1], 0));
                if (p - 2 >= 0 && g->dn_rec[p - 2]) OC_CUDA(cudaStreamWaitEvent(s1, g->ev_down[p - 2], 0));
                const double up0 = S.h2d_bytes;
                rc = trace_begin(u, 0, s1);
                if (rc) return rc;
                if (g->flags & OC_FLAG_MANAGED) {
                    for (const DatPlan& dp : P.dp) {
                        rc = managed_prefetch(dp, g->dats[dp.dat], u, true, s1, S.h2d_bytes);
                        if (rc) return rc;
                    }
                }
                // halo-strip copies of this tile (SM-driven) go to the side stream, forked
                // after the phase's waits and joined before the tile's upload event
                bool strip_side = false;
                for (const DatPlan& dp : P.dp)
                    for (const Interval& iv : dp.up)
                        if (iv.t == u && iv.x0 < iv.x1 && g->dats[dp.dat].host_dev) strip_side = true;
                if (g->flags & OC_FLAG_MANAGED) strip_side = false;
                cudaStream_t ss = strip_side ? g->s1b : s1;
                if (strip_side) {
                    OC_CUDA(cudaEventRecord(g->ev_sf, s1));
                    OC_CUDA(cudaStreamWaitEvent(g->s1b, g->ev_sf, 0));
                }
                StripBatch strips;
                strips.njobs = 0;
                for (size_t di = 0; di < P.dp.size() && !(g->flags & OC_FLAG_MANAGED); ++di) {
                    const DatPlan& dp = P.dp[di];
                    const Dat& d = g->dats[dp.dat];
                    char* slab = g->arena + dp.off;
                    const std::vector<Interval>* have = (u == 0 && pf_match) ? &g->pf.rows[di] : nullptr;
                    for (const Interval& iv : dp.up) {
                        if (iv.t != u) continue;
                        rc = for_missing(iv, have, [&](int a, int b) {
                            return copy_rows(d, slab, dp.S, a, b, true, s1, S.h2d_bytes, iv.x0, iv.x1, nullptr,
                                             &strips, &S, ss);
                        });
                        if (rc) break;
                    }
                    if (rc) break;
                }
                if (!rc) rc = flush_strips(strips, ss, &S);
                if (strip_side) {
                    // joined even after a failure, so that a capture in progress can end
                    cudaEventRecord(g->ev_sj, g->s1b);
                    cudaStreamWaitEvent(s1, g->ev_sj, 0);
                }
                if (rc) return rc;
                rc = trace_end(s1, S.h2d_bytes - up0);
                if (rc) return rc;
                // (an event recorded behind stream waits alone was seen to release its
                // waiters only when the stream's next copy completed: skip it)
                g->up_rec[u] = S.h2d_bytes > up0;
                if (g->up_rec[u]) OC_CUDA(cudaEventRecord(g->ev_up[u], s1));
            }
            if (k == 0 && p >= 0 && p < T) {
                if (g->up_rec[p]) OC_CUDA(cudaStreamWaitEvent(s0, g->ev_up[p], 0));
                if (p - 2 >= 0 && g->dn_rec[p - 2]) OC_CUDA(cudaStreamWaitEvent(s0, g->ev_down[p - 2], 0));
                rc = trace_begin(p, 1, s0);
                if (!rc) rc = run_compute(p);
                if (!rc) rc = trace_end(s0, 0.0);
                if (rc) return rc;
                OC_CUDA(cudaEventRecord(g->ev_comp[p], s0));
            }
            const int q = p - 1;
            if (q >= 0 && q < T) {
                OC_CUDA(cudaStreamWaitEvent(s2, g->ev_comp[q], 0));
                const double dn0 = S.d2h_bytes;
                rc = trace_begin(q, 2, s2);
                if (rc) return rc;
                if ((g->flags & OC_FLAG_MANAGED) && T > 1)
                    for (const DatPlan& dp : P.dp) {
                        rc = managed_prefetch(dp, g->dats[dp.dat], q, false, s2, S.d2h_bytes);
                        if (rc) return rc;
                    }
                for (size_t di = 0; di < P.dp.size() && !(g->flags & OC_FLAG_MANAGED); ++di) {
                    const DatPlan& dp = P.dp[di];
                    const Dat& d = g->dats[dp.dat];
                    for (const Interval& iv : dp.down)
                        if (iv.t == q) {
                            rc = copy_rows(d, g->arena + dp.off, dp.S, iv.a, iv.b, false, s2, S.d2h_bytes, 0, 0,
                                           trial ? g->trial_sink : nullptr);
                            if (rc) return rc;
                        }
                }
                rc = trace_end(s2, S.d2h_bytes - dn0);
                if (rc) return rc;
                g->dn_rec[q] = S.d2h_bytes > dn0;
                if (g->dn_rec[q]) OC_CUDA(cudaEventRecord(g->ev_down[q], s2));
            }
        }
        if (pf_match) S.prefetched_bytes = g->pf.bytes;
        g->pf.active = false;
    }

    // reductions: deterministic fold of the per-row partials
    for (size_t r = 0; r < P.rp.size(); ++r) {
        const RedPlan& rp = P.rp[r];
        double* res = (double*)(g->arena + sb + P.results_off) + r;
        cudaError_t e = launch_combine((const double*)(g->arena + sb + rp.part_off), rp.count, rp.op, res, s0);
        if (e != cudaSuccess) return fail(OC_ERR_CUDA, "combine launch failed: %s", cudaGetErrorString(e));
        S.kernel_launches++;
    }
    if (!P.rp.empty()) {
        OC_CUDA(cudaEventRecord(g->ev_res, s0));
        OC_CUDA(cudaStreamWaitEvent(s2, g->ev_res, 0));
        OC_CUDA(cudaMemcpyAsync(hr, g->arena + sb + P.results_off, P.rp.size() * 8,
                                cudaMemcpyDeviceToHost, s2));
    }
    if (!trial && !P.incore && (g->flags & OC_FLAG_PREFETCH) && !(g->flags & OC_FLAG_MANAGED)) {
        rc = issue_prefetch(P);
        if (rc) return rc;
    }
    return OC_OK;
}

// Wait for a chain issued by run_plan and publish its results and counters.
static int finish_chain(Plan& P, const std::vector<Loop>& loops, bool trial, bool graphed, double* ms_out,
                        oc_stats_t& S, std::chrono::steady_clock::time_point t0, const double* hr)
{
    cudaStream_t s0 = g->st[0];
    int rc = OC_OK;
    (void)loops;
    if (trial) {
        if (!P.incore && P.T > 0 && g->dn_rec[P.T - 1]) OC_CUDA(cudaStreamWaitEvent(s0, g->ev_down[P.T - 1], 0));
        OC_CUDA(cudaEventRecord(g->tm1, s0));
        rc = wait_event(g->tm1, g->timeout_s);
        if (rc) return rc;
        float ms = 0;
        OC_CUDA(cudaEventElapsedTime(&ms, g->tm0, g->tm1));
        if (ms_out) *ms_out = ms;
        return OC_OK;
    }
    rc = wait_stream(s0);
    if (rc) return rc;
    if (!graphed) {   // downloads and the results copy (a whole-chain graph ends on s0)
        rc = wait_stream(g->st[2]);
        if (rc) return rc;
    }
    for (size_t r = 0; r < P.rp.size(); ++r) {
        g->red_val[P.rp[r].handle] = hr[r];
        g->red_has[P.rp[r].handle] = 1;
    }
    if (!g->prof_pending.empty()) {
        rc = collect_profile();
        if (rc) return rc;
    }
    if (!g->tr.empty()) {
        rc = collect_trace();
        if (rc) return rc;
    }
    double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    S.seconds = sec;
    S.total_seconds += sec;
    S.total_cell_updates += S.cell_updates;
    S.total_hbm_bytes += S.hbm_bytes;
    S.total_h2d_bytes += S.h2d_bytes;
    S.total_d2h_bytes += S.d2h_bytes;
    S.total_kernel_launches += S.kernel_launches;
    S.chains++;
    return OC_OK;
}

// The cyclic flag (Sec. 4.1) is a promise that the chain is the one repeated: a dataset
// it writes before reading is a temporary, so a streamed plan never downloads it and its
// host rows keep older values. A later chain that reads such a dataset before writing it
// breaks the promise and would compute from those rows; it is refused instead. A device
// copy that is current (in-core or resident datasets) is the dataset's value and needs no
// host rows, and a managed store is one copy, so neither is affected.
static int cyclic_guard(const Plan& P, const std::vector<Loop>& loops)
{
    const size_t ND = g->dats.size();
    std::vector<uint8_t> first(ND, 0), written(ND, 0);   // first: 1 written first, 2 read first
    for (const Loop& lp : loops) {
        for (const Arg& ar : lp.args)
            if (ar.access != OC_REDUCE && (ar.access == OC_READ || ar.access == OC_RW) && !first[ar.dat])
                first[ar.dat] = 2;
        for (const Arg& ar : lp.args)
            if (ar.access != OC_REDUCE && (ar.access == OC_WRITE || ar.access == OC_RW)) {
                if (!first[ar.dat]) first[ar.dat] = 1;
                written[ar.dat] = 1;
            }
    }
    for (size_t k = 0; k < ND; ++k) {
        const Dat& d = g->dats[k];
        if (first[k] != 2 || !d.cyc_stale || d.managed) continue;
        const bool on_dev = P.incore ? (d.resident && d.dev_valid)
                                     : (P.dat_index[k] >= 0 && P.dp[P.dat_index[k]].resident && d.resident &&
                                        d.dev_valid && d.res_off == P.dp[P.dat_index[k]].off);
        if (!on_dev)
            return fail(OC_ERR_STATE,
                        "dataset %zu is read before it is written, but an earlier chain wrote it first under "
                        "the cyclic flag and did not download it: the chain is not the repeated one", k);
    }
    // a dataset this chain writes is stale afterwards exactly when its download is skipped
    const bool skips = (g->flags & OC_FLAG_CYCLIC) && !P.incore && !(g->flags & OC_FLAG_MANAGED);
    for (size_t k = 0; k < ND; ++k)
        if (written[k])
            g->dats[k].cyc_stale = skips && first[k] == 1 && P.dat_index[k] >= 0 && !P.dp[P.dat_index[k]].resident;
    return OC_OK;
}

static int execute()
{
    if (g->queue.empty()) return OC_OK;
    auto t0 = std::chrono::steady_clock::now();
    std::vector<Loop> loops;
    loops.swap(g->queue);
    Plan* Pp = nullptr;
    int rc = select_plan(loops, Pp);
    if (rc) return rc;
    Plan& P = *Pp;
    g->last = Pp;

    oc_stats_t& S = g->stats;
    S.tiles = P.T;
    S.tile_height = P.h;
    S.depth = P.depth;
    S.resident_dats = P.res_dats;
    S.resident_bytes = (double)P.res_bytes;
    S.loops = P.L;
    S.cell_updates = 0;
    S.hbm_bytes = 0;
    S.h2d_bytes = 0;
    S.d2h_bytes = 0;
    S.prefetched_bytes = 0;
    S.graph_replays = 0;
    S.kernel_launches = 0;
    for (const Loop& lp : loops) {
        double pts = (double)lp.points();
        S.cell_updates += pts;
        for (const Arg& ar : lp.args)
            if (ar.access != OC_REDUCE)
                S.hbm_bytes += pts * g->dats[ar.dat].esz * (ar.access == OC_RW ? 2 : 1);
    }
    rc = cyclic_guard(P, loops);
    if (rc) return rc;
    if (g->dryrun) {
        S.seconds = 0;
        S.chains++;
        return OC_OK;
    }
    rc = run_plan(P, loops, false, nullptr, t0);
    g->trial = false;
    return rc;
}


// ---------------------------------------------------------------------------------
static bool known_kernel(int k) { return (k >= OC_K_COPY && k <= OC_K_HILO_ADD) || physics_kernel_known(k); }

static int validate_loop(Loop& lp)
{
    const int nargs = (int)lp.args.size();
    int ndim = -1, dtype = -1;
    for (const Arg& ar : lp.args)
        if (ar.access != OC_REDUCE) {
            const Dat& d = g->dats[ar.dat];
            if (ndim < 0) ndim = d.ndim;
            if (d.ndim != ndim) return fail(OC_ERR_ARG, "loop mixes 2-D and 3-D datasets");
            if (dtype < 0) dtype = d.dtype;
            if (d.dtype != dtype) return fail(OC_ERR_ARG, "loop mixes element types");
        }
    if (ndim < 0) return fail(OC_ERR_ARG, "loop has no dataset argument");
    lp.ndim = ndim;
    const int sa = ndim - 1;
    for (int a = ndim; a < 3; ++a) { lp.lo[a] = 0; lp.hi[a] = 1; }
    for (Arg& ar : lp.args) {
        if (ar.access == OC_REDUCE) continue;
        const Dat& d = g->dats[ar.dat];
        for (int a = 0; a < 3; ++a) { ar.rmin[a] = 0; ar.rmax[a] = 0; }
        for (size_t p = 0; p < ar.off.size(); ++p)
            for (int a = 0; a < 3; ++a) {
                if (a >= ndim && ar.off[p][a] != 0) return fail(OC_ERR_ARG, "offset on a missing axis");
                if (p == 0 || ar.off[p][a] < ar.rmin[a]) ar.rmin[a] = ar.off[p][a];
                if (p == 0 || ar.off[p][a] > ar.rmax[a]) ar.rmax[a] = ar.off[p][a];
            }
        if (ar.access == OC_WRITE || ar.access == OC_RW) {
            if (ar.off.size() != 1 || ar.off[0][0] || ar.off[0][1] || ar.off[0][2])
                return fail(OC_ERR_ARG, "a written argument must use the single offset 0");
        }
        bool empty = false;
        for (int a = 0; a < ndim; ++a) empty = empty || lp.lo[a] >= lp.hi[a];
        if (empty) continue;
        for (int a = 0; a < ndim; ++a) {
            const bool wrap = (d.periodic & (1 << a)) && a != sa;
            if (wrap) {
                if (lp.lo[a] < 0 || lp.hi[a] > d.size[a] || ar.rmin[a] <= -d.size[a] || ar.rmax[a] >= d.size[a])
                    return fail(OC_ERR_ARG, "periodic axis %d: range or offset out of [0, n)", a);
            } else if (lp.lo[a] + ar.rmin[a] < -d.hlo[a] || lp.hi[a] - 1 + ar.rmax[a] >= d.size[a] + d.hhi[a]) {
                return fail(OC_ERR_ARG, "argument on dataset %d reaches outside its allocated extent on axis %d", ar.dat, a);
            }
        }
    }
    // a dataset written by the loop may not be read at a non-zero offset
    for (const Arg& w : lp.args) {
        if (w.access != OC_WRITE && w.access != OC_RW) continue;
        for (const Arg& r : lp.args) {
            if (r.access != OC_READ || r.dat != w.dat) continue;
            for (auto& o : r.off)
                if (o[0] || o[1] || o[2]) return fail(OC_ERR_ARG, "dataset %d is written and read at a non-zero offset", w.dat);
        }
    }
    auto acc = [&](int j) { return j < nargs ? lp.args[j].access : -1; };
    auto npts = [&](int j) { return (int)lp.args[j].off.size(); };
    switch (lp.kernel) {
    case OC_K_COPY:
        if (nargs != 2 || acc(0) != OC_WRITE || acc(1) != OC_READ || npts(1) != 1)
            return fail(OC_ERR_ARG, "COPY takes [WRITE dst, READ src (1 point)]");
        break;
    case OC_K_LINCOMB: {
        if (nargs < 2 || acc(0) != OC_WRITE) return fail(OC_ERR_ARG, "LINCOMB takes [WRITE dst, READ inputs...]");
        int M = 0;
        for (int j = 1; j < nargs; ++j) {
            if (acc(j) != OC_READ) return fail(OC_ERR_ARG, "LINCOMB inputs must be READ");
            M += npts(j);
        }
        if (M > kLaunchMaxSamples) return fail(OC_ERR_ARG, "LINCOMB supports at most %d samples", kLaunchMaxSamples);
        if ((int)lp.params.size() != 1 + M) return fail(OC_ERR_ARG, "LINCOMB needs 1 + %d parameters", M);
        break;
    }
    case OC_K_REDUCE:
        if ((nargs != 2 && nargs != 3) || acc(nargs - 1) != OC_REDUCE || acc(0) != OC_READ ||
            (nargs == 3 && acc(1) != OC_READ))
            return fail(OC_ERR_ARG, "REDUCE takes [READ src0, (READ src1), REDUCE handle]");
        for (int j = 0; j < nargs - 1; ++j)
            if (npts(j) != 1 || lp.args[j].rmin[0] || lp.args[j].rmin[1] || lp.args[j].rmin[2] ||
                lp.args[j].rmax[0] || lp.args[j].rmax[1] || lp.args[j].rmax[2])
                return fail(OC_ERR_ARG, "REDUCE reads at offset 0 only");
        if (lp.params.size() != 1) return fail(OC_ERR_ARG, "REDUCE needs [mode]");
        break;
    case OC_K_HILO_ADD:
        if (nargs != 3 || acc(0) != OC_RW || acc(1) != OC_RW || acc(2) != OC_READ || npts(2) != 1 || dtype != OC_F32)
            return fail(OC_ERR_ARG, "HILO_ADD takes [RW hi, RW lo, READ du] of F32 datasets");
        if (lp.args[2].rmin[0] || lp.args[2].rmax[0] || lp.args[2].rmin[1] || lp.args[2].rmax[1] ||
            lp.args[2].rmin[2] || lp.args[2].rmax[2])
            return fail(OC_ERR_ARG, "HILO_ADD reads du at offset 0");
        if (lp.params.size() != 1) return fail(OC_ERR_ARG, "HILO_ADD needs [scale]");
        break;
    default: {
        std::string msg;
        if (!physics_validate(lp, g->dats, msg)) return fail(OC_ERR_ARG, "%s", msg.c_str());
    }
    }
    int reds = 0;
    for (const Arg& ar : lp.args) reds += ar.access == OC_REDUCE;
    if (reds > 1) return fail(OC_ERR_ARG, "at most one reduction argument per loop");
    if (reds && lp.kernel != OC_K_REDUCE && !physics_kernel_reduces(lp.kernel))
        return fail(OC_ERR_ARG, "kernel %d has no reduction argument", lp.kernel);
    return OC_OK;
}

}  // namespace oc

// =================================================================================
using namespace oc;

extern "C" {

const char* oc_last_error(void) { return g_err; }

int oc_init(size_t budget, void* arena, size_t arena_bytes, void* const streams[3], uint32_t flags,
            int planner_mode)
{
    if (g) return fail(OC_ERR_STATE, "oc_init: context already exists");
    if (budget == 0) return fail(OC_ERR_ARG, "oc_init: zero budget");
    if (planner_mode < OC_PLAN_FIXED || planner_mode > OC_PLAN_LEARNED) return fail(OC_ERR_ARG, "oc_init: planner mode");
    if (arena && arena_bytes < budget) return fail(OC_ERR_ARG, "oc_init: arena smaller than the budget");
    if (!arena && arena_bytes != 0) return fail(OC_ERR_ARG, "oc_init: arena_bytes without an arena");
    Ctx* c = new Ctx();
    c->flags = flags;
    c->planner_mode = planner_mode;
    c->dryrun = (flags & OC_FLAG_DRYRUN) != 0;
    c->budget = (long long)budget;
    if (const char* t = getenv("OC_TIMEOUT_S")) c->timeout_s = atof(t);
    g = c;
    if (!c->dryrun) {
        int ndev = 0;
        cudaError_t e = cudaGetDeviceCount(&ndev);
        if (e != cudaSuccess || ndev == 0) {
            delete c; g = nullptr;
            return fail(OC_ERR_CUDA, "oc_init: no CUDA device (%s)", cudaGetErrorString(e));
        }
        if (arena) { c->arena = (char*)arena; c->arena_bytes = (long long)arena_bytes; }
        else {
            e = cudaMalloc((void**)&c->arena, budget);
            if (e != cudaSuccess) { delete c; g = nullptr; return fail(OC_ERR_CUDA, "oc_init: arena allocation: %s", cudaGetErrorString(e)); }
            c->own_arena = true;
            c->arena_bytes = (long long)budget;
        }
        if (streams && streams[0] && streams[1] && streams[2]) {
            for (int k = 0; k < 3; ++k) c->st[k] = (cudaStream_t)streams[k];
        } else {
            for (int k = 0; k < 3; ++k) cudaStreamCreateWithFlags(&c->st[k], cudaStreamNonBlocking);
            c->own_streams = true;
        }
        cudaEventCreateWithFlags(&c->ev_pf, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_end, cudaEventDisableTiming);
        cudaEventCreate(&c->tm0);
        cudaEventCreate(&c->tm1);
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_fork2, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_j1, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_j2, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_par, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_res, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_resup, cudaEventDisableTiming);
        kernels_prepare();
        cudaStreamCreateWithFlags(&c->s0b, cudaStreamNonBlocking);
        cudaStreamCreateWithFlags(&c->s1b, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&c->ev_sf, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_sj, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_tf, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_tj, cudaEventDisableTiming);
    }
    return OC_OK;
}

int oc_finalize(void)
{
    if (!g) return fail(OC_ERR_STATE, "oc_finalize: no context");
    if (!g->dryrun) {
        for (int k = 0; k < 3; ++k) if (g->st[k]) cudaStreamSynchronize(g->st[k]);
        if (g->s0b) cudaStreamSynchronize(g->s0b);
        if (g->s1b) cudaStreamSynchronize(g->s1b);
        for (auto& kv : g->graphs) {
            for (auto ge : kv.second.tiles) if (ge) cudaGraphExecDestroy(ge);
            for (auto& v : kv.second.prof) for (auto& pr : v) { cudaEventDestroy(pr.a); cudaEventDestroy(pr.b); }
        }
        for (auto e : g->ev_pool) cudaEventDestroy(e);
        for (auto e : g->tr_pool) cudaEventDestroy(e);
        if (g->tr_t0) cudaEventDestroy(g->tr_t0);
        for (auto e : g->ev_up) cudaEventDestroy(e);
        for (auto e : g->ev_comp) cudaEventDestroy(e);
        for (auto e : g->ev_down) cudaEventDestroy(e);
        if (g->ev_pf) cudaEventDestroy(g->ev_pf);
        if (g->ev_end) cudaEventDestroy(g->ev_end);
        for (auto& kv : g->chain_graphs) {
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
            host_free(kv.second.hp, true);
            host_free(kv.second.hr, true);
        }
        for (cudaEvent_t e : {g->ev_fork, g->ev_fork2, g->ev_j1, g->ev_j2, g->ev_par, g->ev_res, g->ev_resup, g->ev_tf,
                              g->ev_tj, g->ev_sf, g->ev_sj})
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : g->ev_launch) cudaEventDestroy(e);
        if (g->s0b) cudaStreamDestroy(g->s0b);
        if (g->s1b) cudaStreamDestroy(g->s1b);
        if (g->tm0) cudaEventDestroy(g->tm0);
        if (g->tm1) cudaEventDestroy(g->tm1);
        host_free(g->trial_sink, true);
        if (g->own_streams) for (int k = 0; k < 3; ++k) cudaStreamDestroy(g->st[k]);
        if (g->own_arena) cudaFree(g->arena);
    }
    for (Dat& d : g->dats) {
        if (d.managed) cudaFree(d.host);
        else host_free(d.host, d.host_pinned);
    }
    host_free(g->h_params, !g->dryrun);
    host_free(g->h_results, !g->dryrun);
    delete g;
    g = nullptr;
    return OC_OK;
}

int oc_decl_dat(int ndim, const int size[3], const int halo_lo[3], const int halo_hi[3], int dtype,
                const void* host_init, int periodic_mask, int* dat_out)
{
    if (!g) return fail(OC_ERR_STATE, "oc_decl_dat: no context");
    if (!dat_out || !size || !halo_lo || !halo_hi) return fail(OC_ERR_ARG, "oc_decl_dat: null pointer");
    if (ndim != 2 && ndim != 3) return fail(OC_ERR_ARG, "oc_decl_dat: ndim must be 2 or 3");
    if (dtype != OC_F64 && dtype != OC_F32) return fail(OC_ERR_ARG, "oc_decl_dat: dtype");
    Dat d;
    d.ndim = ndim;
    for (int a = 0; a < ndim; ++a) {
        if (size[a] < 1 || halo_lo[a] < 0 || halo_hi[a] < 0) return fail(OC_ERR_ARG, "oc_decl_dat: size/halo");
        d.size[a] = size[a]; d.hlo[a] = halo_lo[a]; d.hhi[a] = halo_hi[a];
        if ((periodic_mask & (1 << a)) && a != ndim - 1 && (halo_lo[a] || halo_hi[a]))
            return fail(OC_ERR_ARG, "oc_decl_dat: a periodic fast axis has no halo");
    }
    d.dtype = dtype;
    d.esz = dtype == OC_F64 ? 8 : 4;
    d.periodic = periodic_mask & ((1 << ndim) - 1);
    d.ox = (int)(align_up((long long)d.hlo[0] * d.esz, 16) / d.esz);
    const long long line = d.ox + d.size[0] + d.hhi[0];
    d.pitch = align_up(line, 128 / d.esz);
    d.ylines = ndim == 3 ? d.ext(1) : 1;
    d.row_elems = d.pitch * d.ylines;
    d.nrows = d.ext(ndim - 1);
    d.y0 = -d.hlo[ndim - 1];
    if (!g->dryrun && (g->flags & OC_FLAG_MANAGED)) {
        void* p = nullptr;
        cudaError_t e = cudaMallocManaged(&p, (size_t)d.bytes(), cudaMemAttachGlobal);
        if (e != cudaSuccess)
            return fail(OC_ERR_NOMEM, "oc_decl_dat: managed allocation of %lld bytes failed: %s", d.bytes(),
                        cudaGetErrorString(e));
        d.host = p;
        d.managed = true;
    } else if (!g->dryrun) {
        d.host = host_alloc((size_t)d.bytes(), true);
        if (!d.host) return fail(OC_ERR_NOMEM, "oc_decl_dat: pinned allocation of %lld bytes failed", d.bytes());
        d.host_pinned = true;
        void* mapped = nullptr;
        if (cudaHostGetDevicePointer(&mapped, d.host, 0) == cudaSuccess) d.host_dev = (char*)mapped;
        else cudaGetLastError();
    }
    if (!g->dryrun) {
        memset(d.host, 0, (size_t)d.bytes());
        if (host_init) {
            const long long ext0 = d.ext(0);
            const char* src = (const char*)host_init;
            char* dst = (char*)d.host;
            for (long long r = 0; r < d.nrows; ++r)
                for (long long l = 0; l < d.ylines; ++l)
                    memcpy(dst + ((r * d.row_elems) + l * d.pitch + d.ox - d.hlo[0]) * d.esz,
                           src + ((r * d.ylines + l) * ext0) * d.esz, (size_t)(ext0 * d.esz));
        }
    }
    d.host_valid = true;
    g->dats.push_back(d);
    *dat_out = (int)g->dats.size() - 1;
    return OC_OK;
}

int oc_decl_reduction(int op, int* red_out)
{
    if (!g) return fail(OC_ERR_STATE, "oc_decl_reduction: no context");
    if (!red_out || op < OC_SUM || op > OC_MIN) return fail(OC_ERR_ARG, "oc_decl_reduction: op");
    g->red_ops.push_back(op);
    g->red_val.push_back(0.0);
    g->red_has.push_back(0);
    *red_out = (int)g->red_ops.size() - 1;
    return OC_OK;
}

int oc_enqueue_loop(int kernel_id, const int range_lo[3], const int range_hi[3], int nargs,
                    const oc_arg* args, const double* params, int nparams)
{
    if (!g) return fail(OC_ERR_STATE, "oc_enqueue_loop: no context");
    if (!known_kernel(kernel_id)) return fail(OC_ERR_ARG, "unknown kernel id %d", kernel_id);
    if (nargs < 1 || nargs > kMaxArgs || !args || !range_lo || !range_hi) return fail(OC_ERR_ARG, "oc_enqueue_loop: arguments");
    if (nparams < 0 || (nparams > 0 && !params)) return fail(OC_ERR_ARG, "oc_enqueue_loop: parameters");
    Loop lp;
    lp.kernel = kernel_id;
    for (int a = 0; a < 3; ++a) { lp.lo[a] = range_lo[a]; lp.hi[a] = range_hi[a]; }
    int ndim = 0;
    for (int j = 0; j < nargs; ++j) {
        const oc_arg& a = args[j];
        Arg ar;
        ar.dat = a.dat;
        ar.access = a.access;
        if (a.access == OC_REDUCE) {
            if (a.dat < 0 || a.dat >= (int)g->red_ops.size()) return fail(OC_ERR_ARG, "bad reduction handle %d", a.dat);
        } else {
            if (a.access != OC_READ && a.access != OC_WRITE && a.access != OC_RW) return fail(OC_ERR_ARG, "bad access mode %d", a.access);
            if (a.dat < 0 || a.dat >= (int)g->dats.size()) return fail(OC_ERR_ARG, "bad dataset handle %d", a.dat);
            ndim = g->dats[a.dat].ndim;
            if (a.npoints < 1 || a.npoints > kLaunchMaxSamples || !a.offsets) return fail(OC_ERR_ARG, "bad stencil");
            for (int p = 0; p < a.npoints; ++p) {
                std::array<int, 3> o = {0, 0, 0};
                for (int q = 0; q < ndim; ++q) o[q] = a.offsets[p * ndim + q];
                ar.off.push_back(o);
            }
        }
        lp.args.push_back(ar);
    }
    for (int i = 0; i < nparams; ++i) lp.params.push_back(params[i]);
    int r = validate_loop(lp);
    if (r) return r;
    g->queue.push_back(std::move(lp));
    return OC_OK;
}

int oc_flush(void)
{
    if (!g) return fail(OC_ERR_STATE, "oc_flush: no context");
    return execute();
}

int oc_reduce(int red, double* out)
{
    if (!g) return fail(OC_ERR_STATE, "oc_reduce: no context");
    if (red < 0 || red >= (int)g->red_ops.size() || !out) return fail(OC_ERR_ARG, "oc_reduce: handle");
    int r = execute();
    if (r) return r;
    if (g->dryrun) return fail(OC_ERR_STATE, "oc_reduce: dry-run context executes nothing");
    if (!g->red_has[red]) return fail(OC_ERR_STATE, "oc_reduce: reduction %d was never computed", red);
    *out = g->red_val[red];
    return OC_OK;
}

int oc_fetch_dat(int dat, void* host_out)
{
    if (!g) return fail(OC_ERR_STATE, "oc_fetch_dat: no context");
    if (dat < 0 || dat >= (int)g->dats.size() || !host_out) return fail(OC_ERR_ARG, "oc_fetch_dat: handle");
    int r = execute();
    if (r) return r;
    if (g->dryrun) return fail(OC_ERR_STATE, "oc_fetch_dat: dry-run context holds no data");
    Dat& d = g->dats[dat];
    if (d.resident && !d.host_valid) {
        OC_CUDA(cudaMemcpyAsync(d.host, g->arena + d.res_off, (size_t)d.bytes(), cudaMemcpyDeviceToHost, g->st[2]));
        r = wait_stream(g->st[2]);
        if (r) return r;
        d.host_valid = true;
    }
    const long long ext0 = d.ext(0);
    char* dst = (char*)host_out;
    const char* src = (const char*)d.host;
    for (long long row = 0; row < d.nrows; ++row)
        for (long long l = 0; l < d.ylines; ++l)
            memcpy(dst + ((row * d.ylines + l) * ext0) * d.esz,
                   src + ((row * d.row_elems) + l * d.pitch + d.ox - d.hlo[0]) * d.esz, (size_t)(ext0 * d.esz));
    // a periodic slow axis: its halo rows are returned as the periodic images of the
    // interior (row y takes row y mod n), whatever the last chain left in them
    const int sa = d.slow();
    if (d.periodic & (1 << sa)) {
        const int n = d.size[sa], lo = d.hlo[sa];
        const size_t rb = (size_t)(d.ylines * ext0 * d.esz);
        for (int y = -lo; y < n + d.hhi[sa]; ++y) {
            if (y >= 0 && y < n) continue;
            const int yi = ((y % n) + n) % n;
            memcpy(dst + (size_t)(y + lo) * rb, dst + (size_t)(yi + lo) * rb, rb);
        }
    }
    return OC_OK;
}

int oc_set_flag(uint32_t flag, int on)
{
    if (!g) return fail(OC_ERR_STATE, "oc_set_flag: no context");
    if (flag & ~(OC_FLAG_CYCLIC | OC_FLAG_PREFETCH | OC_FLAG_GRAPHS | OC_FLAG_PROFILE | OC_FLAG_TRACE))
        return fail(OC_ERR_ARG, "oc_set_flag: flag");
    if (on) g->flags |= flag;
    else g->flags &= ~flag;
    return OC_OK;
}

int oc_set_tiling(int tile_height, int depth)
{
    if (!g) return fail(OC_ERR_STATE, "oc_set_tiling: no context");
    if (tile_height < 0 || depth < 0 || depth == 1 || depth > 4) return fail(OC_ERR_ARG, "oc_set_tiling: values");
    g->force_h = tile_height;
    g->force_depth = depth;
    return OC_OK;
}

int oc_set_residency(double level)
{
    if (!g) return fail(OC_ERR_STATE, "oc_set_residency: no context");
    if (!(level < 1.0)) return fail(OC_ERR_ARG, "oc_set_residency: level must be below 1");
    g->force_res = level < 0 ? -1.0 : level;
    return OC_OK;
}

int oc_stats(oc_stats_t* out)
{
    if (!g) return fail(OC_ERR_STATE, "oc_stats: no context");
    if (!out) return fail(OC_ERR_ARG, "oc_stats: null");
    *out = g->stats;
    return OC_OK;
}

int oc_kernel_stats(int kernel_id, oc_kernel_stats_t* out)
{
    if (!g) return fail(OC_ERR_STATE, "oc_kernel_stats: no context");
    if (!out) return fail(OC_ERR_ARG, "oc_kernel_stats: null");
    auto it = g->kstats.find(kernel_id);
    KStat k = it == g->kstats.end() ? KStat() : it->second;
    out->launches = k.launches;
    out->ms = k.ms;
    out->bytes = k.bytes;
    out->points = k.points;
    return OC_OK;
}

int oc_trace(oc_trace_rec* out, int cap, int* n)
{
    if (!g) return fail(OC_ERR_STATE, "oc_trace: no context");
    if (!n || (cap > 0 && !out)) return fail(OC_ERR_ARG, "oc_trace: null");
    *n = (int)g->tr_out.size();
    for (int i = 0; i < cap && i < *n; ++i) out[i] = g->tr_out[i];
    return OC_OK;
}

int oc_inject_fault(int site, long long after)
{
    if (!g) return fail(OC_ERR_STATE, "oc_inject_fault: no context");
    if (site < 0 || site > 2) return fail(OC_ERR_ARG, "oc_inject_fault: site must be 0, 1 or 2");
    g->fault_after[site] = after < 0 ? -1 : after;
    return OC_OK;
}

int oc_numa_nodes(int dat, int* store_node, int* gpu_host_node)
{
    if (!g) return fail(OC_ERR_STATE, "oc_numa_nodes: no context");
    if (dat < 0 || dat >= (int)g->dats.size() || !store_node || !gpu_host_node)
        return fail(OC_ERR_ARG, "oc_numa_nodes: arguments");
    *store_node = -1;
    *gpu_host_node = -1;
    const Dat& d = g->dats[dat];
#ifdef SYS_get_mempolicy
    if (d.host) {
        int node = -1;
        // MPOL_F_NODE | MPOL_F_ADDR: the node holding the page at the given address
        if (syscall(SYS_get_mempolicy, &node, nullptr, 0UL, d.host, 3UL) == 0) *store_node = node;
    }
#endif
    if (!g->dryrun) {
        int dev = 0, v = -1;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrHostNumaId, dev) == cudaSuccess)
            *gpu_host_node = v;
        else
            cudaGetLastError();
    }
    return OC_OK;
}

int oc_planner_features(float* out8)
{
    if (!g) return fail(OC_ERR_STATE, "oc_planner_features: no context");
    if (!out8) return fail(OC_ERR_ARG, "oc_planner_features: null");
    for (int k = 0; k < 8; ++k) out8[k] = g->features[k];
    return OC_OK;
}

int oc_autotune_result(double* table, int cap, int* n)
{
    if (!g) return fail(OC_ERR_STATE, "oc_autotune_result: no context");
    if (!n || (cap > 0 && !table)) return fail(OC_ERR_ARG, "oc_autotune_result: null");
    *n = (int)g->tune.size();
    for (int i = 0; i < cap && i < *n; ++i)
        for (int k = 0; k < 6; ++k) table[6 * i + k] = g->tune[i][k];
    return OC_OK;
}

int oc_planner_load(const float* params, int nparams, const float* feat_mean, const float* feat_std)
{
    if (!params || !feat_mean || !feat_std || nparams != mlp_nparams())
        return fail(OC_ERR_ARG, "oc_planner_load: expects %d parameters, 8 means and 8 deviations", mlp_nparams());
    planner_load(params, feat_mean, feat_std);
    if (g) g->chosen.clear();
    return OC_OK;
}

int oc_planner_alternatives(const int* alt6)
{
    if (!alt6) return fail(OC_ERR_ARG, "oc_planner_alternatives: null");
    PlanChoice a[2];
    for (int k = 0; k < 2; ++k) {
        a[k] = PlanChoice{alt6[3 * k], alt6[3 * k + 1], alt6[3 * k + 2]};
        if (a[k].grid < 0 || a[k].grid >= kGridN || a[k].depth < 2 || a[k].depth > 4 || a[k].res < 0 ||
            a[k].res >= kResN)
            return fail(OC_ERR_ARG, "oc_planner_alternatives: candidate %d out of the grid", k);
    }
    planner_set_alternatives(a);
    if (g) g->chosen.clear();
    return OC_OK;
}

int oc_mlp_nparams(void) { return mlp_nparams(); }

int oc_mlp_forward(const float* params, const float* X, int n, float* Y)
{
    if (!params || !X || !Y || n < 1) return fail(OC_ERR_ARG, "oc_mlp_forward: arguments");
    cudaError_t e = mlp_forward(params, X, n, Y);
    if (e != cudaSuccess) return fail(OC_ERR_CUDA, "oc_mlp_forward: %s", cudaGetErrorString(e));
    return OC_OK;
}

int oc_mlp_loss_grad(const float* params, const float* X, const float* T, int n, float* grad, double* loss)
{
    if (!params || !X || !T || !grad || n < 1) return fail(OC_ERR_ARG, "oc_mlp_loss_grad: arguments");
    cudaError_t e = mlp_loss_grad(params, X, T, n, grad, loss);
    if (e != cudaSuccess) return fail(OC_ERR_CUDA, "oc_mlp_loss_grad: %s", cudaGetErrorString(e));
    return OC_OK;
}

int oc_mlp_train(float* params, const float* X, const float* T, int n, int epochs, float lr, float* loss_hist)
{
    if (!params || !X || !T || n < 1 || epochs < 0 || !(lr > 0)) return fail(OC_ERR_ARG, "oc_mlp_train: arguments");
    cudaError_t e = mlp_train(params, X, T, n, epochs, lr, loss_hist);
    if (e != cudaSuccess) return fail(OC_ERR_CUDA, "oc_mlp_train: %s", cudaGetErrorString(e));
    return OC_OK;
}

int oc_kernel_stats_reset(void)
{
    if (!g) return fail(OC_ERR_STATE, "oc_kernel_stats_reset: no context");
    g->kstats.clear();
    return OC_OK;
}

int oc_plan_shape(int* ntiles, int* nloops, int* ndats, int* tile_height, int* depth, int* slow_rows)
{
    if (!g) return fail(OC_ERR_STATE, "oc_plan_shape: no context");
    static const Plan empty;
    const Plan& P = g->last ? *g->last : empty;
    if (ntiles) *ntiles = P.T;
    if (nloops) *nloops = P.L;
    if (ndats) *ndats = (int)P.dp.size();
    if (tile_height) *tile_height = P.h;
    if (depth) *depth = P.depth;
    if (slow_rows) *slow_rows = P.Y1 - P.Y0;
    return OC_OK;
}

int oc_plan_ranges(int* se)
{
    if (!g) return fail(OC_ERR_STATE, "oc_plan_ranges: no context");
    if (!se) return fail(OC_ERR_ARG, "oc_plan_ranges: null");
    if (g->last) std::copy(g->last->se.begin(), g->last->se.end(), se);
    return OC_OK;
}

int oc_plan_dat(int k, int* dat, int* slab_rows, int* up, int cap_up, int* nup, int* down, int cap_down,
                int* ndown)
{
    if (!g) return fail(OC_ERR_STATE, "oc_plan_dat: no context");
    if (!g->last) return fail(OC_ERR_STATE, "oc_plan_dat: no plan yet");
    const Plan& P = *g->last;
    if (k < 0 || k >= (int)P.dp.size()) return fail(OC_ERR_ARG, "oc_plan_dat: index");
    const DatPlan& dp = P.dp[k];
    if (dat) *dat = dp.dat;
    if (slab_rows) *slab_rows = dp.S;
    if (nup) *nup = (int)dp.up.size();
    if (ndown) *ndown = (int)dp.down.size();
    if ((int)dp.up.size() > cap_up || (int)dp.down.size() > cap_down)
        return fail(OC_ERR_ARG, "oc_plan_dat: capacity too small");
    auto put = [](int* o, const Interval& iv) { o[0] = iv.t; o[1] = iv.a; o[2] = iv.b; o[3] = iv.x0; o[4] = iv.x1; };
    for (size_t j = 0; j < dp.up.size(); ++j) put(up + 5 * j, dp.up[j]);
    for (size_t j = 0; j < dp.down.size(); ++j) put(down + 5 * j, dp.down[j]);
    return OC_OK;
}

}  // extern "C"
