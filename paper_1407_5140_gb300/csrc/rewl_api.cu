// rewl_api.cu -- host side of the C ABI declared in include/rewl.h.
//
// Builds the geometry of each instance (bins, windows, realisable energies),
// owns the device state, plans the sweep launches (one per size class, run
// concurrently on forked streams; windows per block and lanes per walker from
// the autotuner), captures the sweep/exchange cycle in a CUDA graph, and joins
// the ln g pieces on the host for rewl_get_dos (Sec. II B).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "rewl.h"
#include "rewl_internal.h"

using namespace rewl;
typedef unsigned long long ull;

struct HostInst {
    rewl_instance desc;
    InstDev dev;
    std::vector<int> lo;
    std::vector<int> ww;          // bins of each window (dev.w is the widest)
    std::vector<uint8_t> reach;
    std::vector<int> n_reach;
};

struct SizeClass {
    int model, L, q, w, m, lat_words, N;
    std::vector<int> insts;
    std::vector<WorkItem> items;
    WorkItem *d_items = nullptr;
    SweepLaunch sl{};
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

struct rewl_ctx {
    std::vector<HostInst> inst;
    int n_win = 0, n_slots = 0;
    long long n_lng = 0, n_lat = 0, n_reach_bytes = 0;
    // device buffers
    InstDev *d_inst = nullptr;
    int32_t *d_lo = nullptr, *d_ww = nullptr, *d_nreach = nullptr, *d_stage = nullptr;
    uint8_t *d_conv = nullptr;
    int64_t *d_conv_sweep = nullptr;
    ull *d_ex_prop = nullptr, *d_ex_acc = nullptr;
    int64_t *d_stage_sweep = nullptr;
    int32_t *d_cfg = nullptr, *d_E = nullptr, *d_bin = nullptr, *d_replica = nullptr, *d_slot_inst = nullptr;
    ull *d_draw = nullptr, *d_nacc = nullptr;
    uint8_t *d_latch = nullptr;
    long long *d_lng = nullptr, *d_lng0 = nullptr;
    uint32_t *d_H = nullptr, *d_lat = nullptr;
    uint8_t *d_reach = nullptr;
    ull *d_counters = nullptr;
    int *d_error = nullptr;
    ExTask *d_ex0 = nullptr, *d_ex1 = nullptr;
    int n_ex0 = 0, n_ex1 = 0;
    DevState st{};
    std::vector<SizeClass> classes;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaEvent_t fork = nullptr;
    long check_every = 1;
    long max_sweeps_per_launch = 1L << 30;
    int force_producers = 0, force_wpc = 0;
    int lattice_mode = 0;               // 0: by size, 1: global memory, 2: shared memory
    int shift_exp = 20;                 // a running window's ln g is lowered by 2^shift_exp once all of it reaches that
    int tune_mode = 1;                  // 1: measure candidate shapes, 0: rule only
    int tune_target = 0, tune_bias = 0; // chosen walkers-per-block target / producer bias
    bool planned = false;
    cudaGraphExec_t graph = nullptr;
    long graph_sweeps = -1;
    long graph_launches = 0;
    long launches = 0;
    long long bytes_h2d = 0, bytes_d2h = 0;   // host<->device bytes the library copied
    int failed = 0;
    std::string err;
};

static thread_local std::string g_create_error;

// Largest lattice side (the site -> (row, column) division by a multiply-high
// with ceil(2^32 / L) is exact for every site of an L x L lattice while
// L^3 < 2^32); lattices above kSharedLatticeBytes per walker stay in global
// memory during sweeps (Potts L > 128, Ising L > 352).
static const int kMaxL = 512;
static const long long kSharedLatticeBytes = 16384;

static rewl_status fail(rewl_ctx *c, rewl_status s, const std::string &msg)
{
    if (c) {
        if (!c->failed) c->err = msg;
        if (s == REWL_ECUDA || s == REWL_EDEVICE) c->failed = 1;
    } else {
        g_create_error = msg;
    }
    return s;
}

// Every host<->device copy of a context goes through these, which count its
// bytes (rewl_transfer_bytes).
static cudaError_t h2d(rewl_ctx *ctx, void *dst, const void *src, size_t n, cudaStream_t s)
{
    ctx->bytes_h2d += (long long)n;
    return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s);
}

static cudaError_t h2d_sync(rewl_ctx *ctx, void *dst, const void *src, size_t n)
{
    ctx->bytes_h2d += (long long)n;
    return cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice);
}

static cudaError_t d2h(rewl_ctx *ctx, void *dst, const void *src, size_t n)
{
    ctx->bytes_d2h += (long long)n;
    return cudaMemcpy(dst, src, n, cudaMemcpyDeviceToHost);
}

#define CK(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(ctx, REWL_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// ---------------------------------------------------------------------------
// geometry (Sec. II A, Fig. 1)
// ---------------------------------------------------------------------------
static bool realisable(int model, int q, long long N, long long E)
{
    const long long off = E + 2 * N;
    if (model == REWL_ISING) {
        if (off < 0 || off > 4 * N || off % 4) return false;
        const long long u = off / 4;  // unsatisfied bonds / 2
        return u != 1 && u != N - 1;
    }
    if (off < 0 || off > 2 * N) return false;
    if (q == 2) return off % 2 == 0 && off != 2 && off != 2 * N - 2;
    return !(off == 1 || off == 2 || off == 3 || off == 5);
}

static rewl_status build_instance(const rewl_instance &d, HostInst &hi, std::string &why,
                                  const int32_t *clo = nullptr, const int32_t *chi = nullptr)
{
    char buf[256];
    if (d.model != REWL_ISING && d.model != REWL_POTTS) { why = "model must be REWL_ISING or REWL_POTTS"; return REWL_EINVAL; }
    if (d.L < 4 || d.L > kMaxL || d.L % 2) { why = "L must be even, 4 <= L <= 512"; return REWL_EINVAL; }
    const int q = d.model == REWL_ISING ? 2 : d.q;
    if (d.model == REWL_POTTS && (q < 2 || q > 127)) { why = "q must be in 2..127"; return REWL_EINVAL; }
    if (d.n_windows < 1 || d.n_windows > 65535) { why = "n_windows must be in 1..65535"; return REWL_EINVAL; }
    if (d.walkers_per_window < 1 || d.walkers_per_window > 32) { why = "walkers_per_window must be in 1..32"; return REWL_EINVAL; }
    if (!(d.overlap >= 0.0 && d.overlap < 1.0)) { why = "overlap must be in [0, 1)"; return REWL_EINVAL; }
    if (d.flat_rule != 0 && d.flat_rule != 1) { why = "flat_rule must be 0 (fraction of mean) or 1 (Zhou-Bhatt)"; return REWL_EINVAL; }
    if (d.flat_rule == 0 && !(d.flatness > 0.0 && d.flatness <= 1.0)) { why = "flatness must be in (0, 1]"; return REWL_EINVAL; }
    if (d.flat_rule == 1 && !(d.flatness > 0.0 && d.flatness <= 1e6)) { why = "Zhou-Bhatt a must be in (0, 1e6]"; return REWL_EINVAL; }
    if (!(d.ln_f_final >= std::ldexp(1.0, -32) && d.ln_f_final <= 1.0)) { why = "ln_f_final must be in [2^-32, 1]"; return REWL_EINVAL; }
    const long long N = (long long)d.L * d.L;
    const int step = d.model == REWL_ISING ? 4 : 1;
    const long long emin_m = -2 * N, emax_m = d.model == REWL_ISING ? 2 * N : 0;
    if (d.e_min < emin_m || d.e_max > emax_m || d.e_min >= d.e_max || (d.e_min - emin_m) % step ||
        (d.e_max - emin_m) % step) {
        snprintf(buf, sizeof buf, "energy range [%lld, %lld] must lie in [%lld, %lld] on the bin grid (step %d)",
                 (long long)d.e_min, (long long)d.e_max, emin_m, emax_m, step);
        why = buf;
        return REWL_EINVAL;
    }
    const int B = (int)((d.e_max - d.e_min) / step) + 1;
    const int h = d.n_windows;
    // equal widths: consecutive windows start (1 - o) w apart and cover B bins
    const double span = 1.0 + (double)(h - 1) * (1.0 - d.overlap);
    int w = (int)std::ceil((double)B / span);
    if (w > B) w = B;
    const int maxdb = d.model == REWL_ISING ? 2 : 4;
    if (!clo && w < 2 * maxdb + 1) { why = "windows narrower than 2 * (largest bin change) + 1"; return REWL_EINVAL; }
    hi.desc = d;
    hi.lo.resize(h);
    hi.ww.assign(h, w);
    for (int i = 0; i < h; ++i) hi.lo[i] = h == 1 ? 0 : (int)(((long long)i * (B - w)) / (h - 1));
    if (clo) {
        // windows given bin by bin (run-time-balanced windows, Sec. V): from bin 0
        // to bin B - 1, increasing ends, each overlapping the next
        if (clo[0] != 0 || chi[h - 1] != B - 1) { why = "windows must start at bin 0 and end at bin B - 1"; return REWL_EINVAL; }
        w = 0;
        for (int i = 0; i < h; ++i) {
            if (chi[i] < clo[i] || chi[i] >= B) { why = "window " + std::to_string(i) + " is empty or past bin B - 1"; return REWL_EINVAL; }
            if (i + 1 < h && (clo[i + 1] <= clo[i] || chi[i + 1] <= chi[i] || clo[i + 1] > chi[i])) {
                why = "windows " + std::to_string(i) + " and " + std::to_string(i + 1) + " must overlap with increasing ends";
                return REWL_EINVAL;
            }
            hi.lo[i] = clo[i];
            hi.ww[i] = chi[i] - clo[i] + 1;
            if (hi.ww[i] < 2 * maxdb + 1) { why = "windows narrower than 2 * (largest bin change) + 1"; return REWL_EINVAL; }
            w = std::max(w, hi.ww[i]);
        }
    }
    hi.reach.resize(B);
    for (int b = 0; b < B; ++b) hi.reach[b] = realisable(d.model, q, N, d.e_min + (long long)b * step);
    hi.n_reach.assign(h, 0);
    for (int i = 0; i < h; ++i)
        for (int b = hi.lo[i]; b < hi.lo[i] + hi.ww[i]; ++b) hi.n_reach[i] += hi.reach[b];
    for (int i = 0; i < h; ++i)
        if (hi.n_reach[i] == 0) { why = "a window holds no realisable energy"; return REWL_EINVAL; }
    int kf = 0;
    while (std::ldexp(1.0, -kf) > d.ln_f_final) ++kf;
    InstDev &I = hi.dev;
    memset(&I, 0, sizeof I);
    I.model = d.model;
    I.L = d.L;
    I.q = q;
    I.N = (int)N;
    I.wpr = d.model == REWL_ISING ? (d.L + 31) / 32 : 0;
    I.lat_words = d.model == REWL_ISING ? d.L * I.wpr : (int)((N + 3) / 4);
    I.magic_L = (uint32_t)((0x100000000ull + (ull)d.L - 1) / (ull)d.L);
    I.step = step;
    I.e_min = d.e_min;
    I.B = B;
    I.h = h;
    I.m = d.walkers_per_window;
    I.w = w;
    I.stage_final = kf;
    I.key0 = (uint32_t)d.seed;
    I.key1 = (uint32_t)(d.seed >> 32) ^ d.instance_id;
    I.p_flat = d.flatness;
    I.flat_rule = d.flat_rule;
    return REWL_OK;
}

// ---------------------------------------------------------------------------
// creation
// ---------------------------------------------------------------------------
template <class T>
static cudaError_t dalloc(T **p, size_t n)
{
    return cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
}

extern "C" void rewl_destroy(rewl_ctx *ctx);
static rewl_status plan(rewl_ctx *ctx);

static rewl_status create_batch(rewl_ctx **out, const rewl_instance *inst, int n_inst, const int32_t *lo,
                                const int32_t *hi, void *cuda_stream);

extern "C" rewl_status rewl_create_batch(rewl_ctx **out, const rewl_instance *inst, int n_inst, void *cuda_stream)
{
    return create_batch(out, inst, n_inst, nullptr, nullptr, cuda_stream);
}

extern "C" rewl_status rewl_create_batch_windows(rewl_ctx **out, const rewl_instance *inst, int n_inst,
                                                 const int32_t *lo, const int32_t *hi, void *cuda_stream)
{
    if (!lo || !hi) return fail(nullptr, REWL_EINVAL, "rewl_create_batch_windows: lo or hi is NULL");
    return create_batch(out, inst, n_inst, lo, hi, cuda_stream);
}

static rewl_status create_batch(rewl_ctx **out, const rewl_instance *inst, int n_inst, const int32_t *lo,
                                const int32_t *hi, void *cuda_stream)
{
    if (!out || !inst || n_inst < 1) return fail(nullptr, REWL_EINVAL, "rewl_create_batch: null argument or n_inst < 1");
    *out = nullptr;
    rewl_ctx *ctx = new rewl_ctx();
    ctx->inst.resize(n_inst);
    long long woff = 0;
    for (int k = 0; k < n_inst; ++k) {
        std::string why;
        if (inst[k].n_windows < 1 || inst[k].n_windows > 65535) {
            delete ctx;
            return fail(nullptr, REWL_EINVAL, "instance " + std::to_string(k) + ": n_windows must be in 1..65535");
        }
        rewl_status s = build_instance(inst[k], ctx->inst[k], why, lo ? lo + woff : nullptr, hi ? hi + woff : nullptr);
        woff += inst[k].n_windows;
        if (s != REWL_OK) {
            delete ctx;
            return fail(nullptr, s, "instance " + std::to_string(k) + ": " + why);
        }
    }
    // offsets
    long long lng = 0, lat = 0, rch = 0;
    int win = 0, slot = 0;
    std::vector<int32_t> lo_all, ww_all, nreach_all, slot_inst;
    std::vector<uint8_t> reach_all;
    std::vector<ExTask> ex0, ex1;
    for (int k = 0; k < n_inst; ++k) {
        HostInst &h = ctx->inst[k];
        InstDev &I = h.dev;
        I.win0 = win;
        I.slot0 = slot;
        I.lng_off = lng;
        I.lat_off = lat;
        I.reach_off = (int)rch;
        const int nw = I.h * I.m;
        win += I.h;
        slot += nw;
        lng += (long long)nw * I.w;
        lat += (long long)nw * I.lat_words;
        rch += I.B;
        for (int i = 0; i < I.h; ++i) {
            lo_all.push_back(h.lo[i]);
            ww_all.push_back(h.ww[i]);
            nreach_all.push_back(h.n_reach[i]);
        }
        reach_all.insert(reach_all.end(), h.reach.begin(), h.reach.end());
        for (int s = 0; s < nw; ++s) slot_inst.push_back(k);
        for (int p = 0; p < 2; ++p)
            for (int i = p; i + 1 < I.h; i += 2)
                for (int j = 0; j < I.m; ++j) (p ? ex1 : ex0).push_back(ExTask{k, i, j, 0});
    }
    ctx->n_win = win;
    ctx->n_slots = slot;
    ctx->n_lng = lng;
    ctx->n_lat = lat;
    ctx->n_reach_bytes = rch;
    ctx->n_ex0 = (int)ex0.size();
    ctx->n_ex1 = (int)ex1.size();
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    *out = ctx;  // from here on errors leave a context the caller destroys
    std::vector<InstDev> idev;
    for (auto &h : ctx->inst) idev.push_back(h.dev);
    CK(dalloc(&ctx->d_inst, n_inst));
    CK(dalloc(&ctx->d_lo, win));
    CK(dalloc(&ctx->d_ww, win));
    CK(dalloc(&ctx->d_nreach, win));
    CK(dalloc(&ctx->d_stage, win));
    CK(dalloc(&ctx->d_conv, win));
    CK(dalloc(&ctx->d_conv_sweep, win));
    CK(dalloc(&ctx->d_ex_prop, win));
    CK(dalloc(&ctx->d_ex_acc, win));
    CK(dalloc(&ctx->d_stage_sweep, (size_t)win * kMaxStages));
    CK(dalloc(&ctx->d_cfg, slot));
    CK(dalloc(&ctx->d_E, slot));
    CK(dalloc(&ctx->d_bin, slot));
    CK(dalloc(&ctx->d_replica, slot));
    CK(dalloc(&ctx->d_slot_inst, slot));
    CK(dalloc(&ctx->d_draw, slot));
    CK(dalloc(&ctx->d_nacc, slot));
    CK(dalloc(&ctx->d_latch, slot));
    CK(dalloc(&ctx->d_lng, lng));
    CK(dalloc(&ctx->d_lng0, lng));
    CK(dalloc(&ctx->d_H, lng));
    CK(dalloc(&ctx->d_lat, lat));
    CK(dalloc(&ctx->d_reach, rch));
    CK(dalloc(&ctx->d_counters, 2));
    CK(dalloc(&ctx->d_error, 1));
    CK(dalloc(&ctx->d_ex0, ex0.size()));
    CK(dalloc(&ctx->d_ex1, ex1.size()));
    cudaStream_t s = ctx->stream;
    CK(h2d(ctx, ctx->d_inst, idev.data(), sizeof(InstDev) * n_inst, s));
    CK(h2d(ctx, ctx->d_lo, lo_all.data(), 4 * win, s));
    CK(h2d(ctx, ctx->d_ww, ww_all.data(), 4 * win, s));
    CK(h2d(ctx, ctx->d_nreach, nreach_all.data(), 4 * win, s));
    CK(h2d(ctx, ctx->d_reach, reach_all.data(), rch, s));
    CK(h2d(ctx, ctx->d_slot_inst, slot_inst.data(), 4 * slot, s));
    if (!ex0.empty()) CK(h2d(ctx, ctx->d_ex0, ex0.data(), sizeof(ExTask) * ex0.size(), s));
    if (!ex1.empty()) CK(h2d(ctx, ctx->d_ex1, ex1.data(), sizeof(ExTask) * ex1.size(), s));
    CK(cudaMemsetAsync(ctx->d_stage, 0, 4 * win, s));
    CK(cudaMemsetAsync(ctx->d_conv, 0, win, s));
    CK(cudaMemsetAsync(ctx->d_conv_sweep, 0xFF, 8 * win, s));
    CK(cudaMemsetAsync(ctx->d_ex_prop, 0, 8 * win, s));
    CK(cudaMemsetAsync(ctx->d_ex_acc, 0, 8 * win, s));
    CK(cudaMemsetAsync(ctx->d_stage_sweep, 0xFF, 8 * (size_t)win * kMaxStages, s));
    CK(cudaMemsetAsync(ctx->d_lng, 0, 8 * lng, s));
    CK(cudaMemsetAsync(ctx->d_lng0, 0, 8 * lng, s));
    CK(cudaMemsetAsync(ctx->d_H, 0, 4 * lng, s));
    CK(cudaMemsetAsync(ctx->d_counters, 0, 16, s));
    CK(cudaMemsetAsync(ctx->d_error, 0, 4, s));
    DevState &st = ctx->st;
    st.inst = ctx->d_inst;
    st.lo = ctx->d_lo;
    st.ww = ctx->d_ww;
    st.n_reach = ctx->d_nreach;
    st.stage = ctx->d_stage;
    st.conv = ctx->d_conv;
    st.conv_sweep = ctx->d_conv_sweep;
    st.ex_prop = ctx->d_ex_prop;
    st.ex_acc = ctx->d_ex_acc;
    st.stage_sweep = reinterpret_cast<long long *>(ctx->d_stage_sweep);
    st.cfg = ctx->d_cfg;
    st.E = ctx->d_E;
    st.bin = ctx->d_bin;
    st.draw = ctx->d_draw;
    st.latch = ctx->d_latch;
    st.n_acc = ctx->d_nacc;
    st.replica = ctx->d_replica;
    st.lng = ctx->d_lng;
    st.lng0 = ctx->d_lng0;
    st.H = ctx->d_H;
    st.lat = ctx->d_lat;
    st.reach = ctx->d_reach;
    st.counters = ctx->d_counters;
    st.error = ctx->d_error;
    CK(cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming));
    int e = launch_init(st, slot, ctx->d_slot_inst, s);
    ctx->launches += 1;
    if (e) return fail(ctx, REWL_ECUDA, std::string("init launch: ") + cudaGetErrorString((cudaError_t)e));
    CK(cudaStreamSynchronize(s));
    int herr = 0;
    CK(d2h(ctx, &herr, ctx->d_error, 4));
    if (herr) return fail(ctx, REWL_EDEVICE, "init: a walker did not reach its window");
    return REWL_OK;
}

extern "C" rewl_status rewl_create(rewl_ctx **out, rewl_model model, int L, int q, long e_min, long e_max,
                                   int n_windows, double overlap, int walkers_per_window, double flatness,
                                   double ln_f_final, unsigned long long seed, void *cuda_stream)
{
    rewl_instance d;
    memset(&d, 0, sizeof d);
    d.model = model;
    d.L = L;
    d.q = q;
    d.n_windows = n_windows;
    d.e_min = e_min;
    d.e_max = e_max;
    d.overlap = overlap;
    d.walkers_per_window = walkers_per_window;
    d.flatness = flatness;
    d.ln_f_final = ln_f_final;
    d.seed = seed;
    d.instance_id = 0;
    return rewl_create_batch(out, &d, 1, cuda_stream);
}

extern "C" void rewl_destroy(rewl_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    for (auto &c : ctx->classes) {
        if (c.d_items) cudaFree(c.d_items);
        if (c.stream) cudaStreamDestroy(c.stream);
        if (c.done) cudaEventDestroy(c.done);
    }
    void *bufs[] = {ctx->d_inst, ctx->d_lo, ctx->d_ww, ctx->d_nreach, ctx->d_stage, ctx->d_conv, ctx->d_conv_sweep,
                    ctx->d_ex_prop, ctx->d_ex_acc, ctx->d_stage_sweep, ctx->d_cfg, ctx->d_E, ctx->d_bin, ctx->d_replica,
                    ctx->d_slot_inst, ctx->d_draw, ctx->d_nacc, ctx->d_latch, ctx->d_lng, ctx->d_lng0, ctx->d_H,
                    ctx->d_lat, ctx->d_reach, ctx->d_counters, ctx->d_error, ctx->d_ex0, ctx->d_ex1};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (ctx->fork) cudaEventDestroy(ctx->fork);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

// ---------------------------------------------------------------------------
// launch planning: one sweep launch per size class; the autotuner fills in
// windows per block and lanes per walker (rewl_tune.cu)
// ---------------------------------------------------------------------------

void rewl::plan_class(rewl_ctx *ctx, int ci, int wpc, int producers)
{
    SizeClass &c = ctx->classes[ci];
    c.items.clear();
    for (int k : c.insts) {
        const InstDev &I = ctx->inst[k].dev;
        const HostInst &hi = ctx->inst[k];
        for (int w0 = 0; w0 < I.h; w0 += wpc) {
            const int n = std::min(wpc, I.h - w0);
            int wrow = 0;
            for (int i = w0; i < w0 + n; ++i) wrow = std::max(wrow, hi.ww[i]);
            c.items.push_back(WorkItem{k, w0, n, wrow});
        }
    }
    const int nw = wpc * c.m;
    c.sl.n_items = (int)c.items.size();
    c.sl.producers = producers;
    c.sl.threads = 32 * (1 + producers);
    c.sl.smem = sweep_smem_bytes(nw, wpc, c.w, c.lat_words, producers, c.N);
    c.sl.max_walkers = nw;
    c.sl.max_w = c.w;
    c.sl.max_lat_words = c.lat_words;
    c.sl.max_win = wpc;
    c.sl.model = c.model;
}

int rewl::class_count(const rewl_ctx *ctx) { return (int)ctx->classes.size(); }
int rewl::class_walkers(const rewl_ctx *ctx, int ci)
{
    int n = 0;
    for (int k : ctx->classes[ci].insts) n += ctx->inst[k].dev.h * ctx->inst[k].dev.m;
    return n;
}
void rewl::class_shape(const rewl_ctx *ctx, int ci, int *model, int *N, int *w, int *m, int *lat_words)
{
    const SizeClass &c = ctx->classes[ci];
    *model = c.model;
    *N = c.N;
    *w = c.w;
    *m = c.m;
    *lat_words = c.lat_words;
}
int rewl::total_walkers(const rewl_ctx *ctx) { return ctx->n_slots; }
int rewl::forced_producers(const rewl_ctx *ctx) { return ctx->force_producers; }
int rewl::forced_wpc(const rewl_ctx *ctx) { return ctx->force_wpc; }
int rewl::tune_target(const rewl_ctx *ctx) { return ctx->tune_target; }
int rewl::tune_producer_bias(const rewl_ctx *ctx) { return ctx->tune_bias; }

// Time a few launch shapes on a shadow context built from the same
// descriptors (its own memory and stream; the caller's walkers are not
// touched) and keep the fastest.  Results do not depend on the shape.
static void measure_shapes(rewl_ctx *ctx)
{
    if (ctx->tune_mode != 1 || ctx->force_wpc || ctx->force_producers) return;
    std::vector<rewl_instance> desc;
    long long trials = 0;
    for (auto &h : ctx->inst) {
        desc.push_back(h.desc);
        trials += (long long)h.dev.h * h.dev.m * h.dev.N;
    }
    const long sweeps = std::max(3L, std::min(50L, (long)(40000000LL / std::max(1LL, trials))));
    const int targets[] = {4, 8, 16, 32};
    const int biases[] = {0, 1};
    float best = 0.f;
    for (int t : targets)
        for (int b : biases) {
            rewl_ctx *sh = nullptr;
            if (rewl_create_batch(&sh, desc.data(), (int)desc.size(), nullptr) != REWL_OK) {
                rewl_destroy(sh);
                return;
            }
            sh->tune_mode = 0;
            sh->tune_target = t;
            sh->tune_bias = b;
            sh->lattice_mode = ctx->lattice_mode;
            sh->shift_exp = ctx->shift_exp;
            sh->check_every = ctx->check_every;
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            float ms = -1.f;
            if (rewl_run(sh, 1) == REWL_OK && cudaEventCreate(&e0) == cudaSuccess &&
                cudaEventCreate(&e1) == cudaSuccess && cudaEventRecord(e0, sh->stream) == cudaSuccess &&
                rewl_run(sh, sweeps) == REWL_OK && cudaEventRecord(e1, sh->stream) == cudaSuccess &&
                cudaEventSynchronize(e1) == cudaSuccess)
                cudaEventElapsedTime(&ms, e0, e1);
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            rewl_destroy(sh);
            if (ms > 0.f && (best == 0.f || ms < best)) {
                best = ms;
                ctx->tune_target = t;
                ctx->tune_bias = b;
            }
        }
    cudaGetLastError();
}

// Blocks whose windows are narrower than the instance's widest need shorter
// ln g rows in shared memory: split each size class into launches by the
// block row width (rounded up to 64 bins), each asking only for the shared
// memory its widest block needs, and give each launch the block shape its
// rows allow (adjacent window groups of one instance merged into larger
// blocks where narrow rows leave the room).  Equal-width windows stay one
// launch.
static void split_by_row(rewl_ctx *ctx)
{
    std::vector<SizeClass> out;
    for (auto &c : ctx->classes) {
        std::map<int, std::vector<WorkItem>> by;
        for (const WorkItem &it : c.items) by[std::min(c.w, (it.wrow + 63) / 64 * 64)].push_back(it);
        if (by.size() <= 1) {
            out.push_back(c);
            continue;
        }
        for (auto &kv : by) {
            SizeClass d = c;
            int wmax = 0, wpc = 0;
            for (const WorkItem &it : kv.second) {
                wmax = std::max(wmax, it.wrow);
                wpc = std::max(wpc, it.n_win);
            }
            int wpc2 = 0, prod2 = 0;
            if (!rewl::block_shape(ctx, c.model, c.N, wmax, c.m, c.lat_words, &wpc2, &prod2) && wpc2 > wpc) {
                // merge runs of adjacent windows of one instance up to wpc2 windows
                std::vector<WorkItem> merged;
                for (const WorkItem &it : kv.second) {
                    if (!merged.empty()) {
                        WorkItem &bk = merged.back();
                        if (bk.inst == it.inst && bk.win_begin + bk.n_win == it.win_begin &&
                            bk.n_win + it.n_win <= wpc2) {
                            bk.n_win += it.n_win;
                            bk.wrow = std::max(bk.wrow, it.wrow);
                            continue;
                        }
                    }
                    merged.push_back(it);
                }
                wpc = 0;
                for (const WorkItem &it : merged) wpc = std::max(wpc, it.n_win);
                d.items = merged;
                d.sl.producers = prod2;
                d.sl.threads = 32 * (1 + prod2);
            } else {
                d.items = kv.second;
            }
            d.sl.n_items = (int)d.items.size();
            d.sl.smem = sweep_smem_bytes(wpc * c.m, wpc, wmax, c.lat_words, d.sl.producers, c.N);
            d.sl.max_w = wmax;
            d.sl.max_walkers = wpc * c.m;
            d.sl.max_win = wpc;
            out.push_back(d);
        }
    }
    ctx->classes.swap(out);
}

static rewl_status plan(rewl_ctx *ctx)
{
    if (ctx->planned) return REWL_OK;
    measure_shapes(ctx);
    std::map<std::vector<int>, int> key2c;
    for (int k = 0; k < (int)ctx->inst.size(); ++k) {
        const InstDev &I = ctx->inst[k].dev;
        std::vector<int> key = {I.model, I.L, I.q, I.w, I.m};
        auto f = key2c.find(key);
        if (f == key2c.end()) {
            SizeClass c;
            c.model = I.model;
            c.L = I.L;
            c.q = I.q;
            c.w = I.w;
            c.m = I.m;
            c.N = I.N;
            // lattices larger than kSharedLatticeBytes stay in global memory
            // (lat_words counts the words a walker keeps in shared memory)
            const bool glat = ctx->lattice_mode == 1 ||
                              (ctx->lattice_mode == 0 && 4LL * I.lat_words > kSharedLatticeBytes);
            c.lat_words = glat ? 0 : I.lat_words;
            c.sl.glat = glat ? 1 : 0;
            ctx->classes.push_back(c);
            f = key2c.emplace(key, (int)ctx->classes.size() - 1).first;
        }
        ctx->classes[f->second].insts.push_back(k);
    }
    if (autotune_plan(ctx)) return fail(ctx, REWL_EINVAL, "no launch configuration fits a window's walkers in shared memory");
    split_by_row(ctx);
    // launch the classes with the largest blocks first: the block scheduler then
    // packs the smaller blocks into the shared memory the large ones leave free
    std::stable_sort(ctx->classes.begin(), ctx->classes.end(),
                     [](const SizeClass &a, const SizeClass &b) { return a.sl.smem > b.sl.smem; });
    for (auto &c : ctx->classes) {
        if (c.sl.smem > 227 * 1024) return fail(ctx, REWL_EINVAL, "window state exceeds shared memory");
        CK(dalloc(&c.d_items, c.items.size()));
        CK(h2d_sync(ctx, c.d_items, c.items.data(), sizeof(WorkItem) * c.items.size()));
        c.sl.items = c.d_items;
        CK(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming));
    }
    // one kernel per model and lattice placement serves every class of that
    // kind: allow the largest dynamic shared memory any of them needs
    for (int kind = 0; kind < 4; ++kind) {
        const int model = kind >> 1, glat = kind & 1;
        int smem = 0;
        for (auto &c : ctx->classes)
            if (c.model == model && c.sl.glat == glat) smem = std::max(smem, c.sl.smem);
        if (!smem) continue;
        int e = prepare_sweep(model, glat != 0, smem);
        if (e) return fail(ctx, REWL_ECUDA, std::string("sweep kernel attributes: ") + cudaGetErrorString((cudaError_t)e));
    }
    ctx->planned = true;
    return REWL_OK;
}

// ---------------------------------------------------------------------------
// running
// ---------------------------------------------------------------------------
static rewl_status check_usable(rewl_ctx *ctx)
{
    if (!ctx) return REWL_EINVAL;
    if (ctx->failed) return REWL_ESTATE;
    return REWL_OK;
}

static rewl_status enqueue_sweeps(rewl_ctx *ctx, long n)
{
    cudaStream_t s = ctx->stream;
    while (n > 0) {
        const long chunk = std::min(n, ctx->max_sweeps_per_launch);
        if (ctx->classes.size() == 1) {
            int e = launch_sweeps(ctx->st, ctx->classes[0].sl, chunk, ctx->check_every, ctx->shift_exp, s);
            if (e) return fail(ctx, REWL_ECUDA, std::string("sweep launch: ") + cudaGetErrorString((cudaError_t)e));
        } else {
            CK(cudaEventRecord(ctx->fork, s));
            for (auto &c : ctx->classes) {
                CK(cudaStreamWaitEvent(c.stream, ctx->fork, 0));
                int e = launch_sweeps(ctx->st, c.sl, chunk, ctx->check_every, ctx->shift_exp, c.stream);
                if (e) return fail(ctx, REWL_ECUDA, std::string("sweep launch: ") + cudaGetErrorString((cudaError_t)e));
                CK(cudaEventRecord(c.done, c.stream));
                CK(cudaStreamWaitEvent(s, c.done, 0));
            }
        }
        int e = launch_bump(ctx->st, chunk, 0, s);
        if (e) return fail(ctx, REWL_ECUDA, std::string("counter launch: ") + cudaGetErrorString((cudaError_t)e));
        ctx->launches += (long)ctx->classes.size() + 1;
        n -= chunk;
    }
    return REWL_OK;
}

static rewl_status enqueue_exchange(rewl_ctx *ctx)
{
    if (ctx->n_ex0 + ctx->n_ex1 > 0) {
        int e = launch_exchange(ctx->st, ctx->d_ex0, ctx->n_ex0, ctx->d_ex1, ctx->n_ex1, ctx->stream);
        if (e) return fail(ctx, REWL_ECUDA, std::string("exchange launch: ") + cudaGetErrorString((cudaError_t)e));
        ctx->launches += 1;
    }
    int e = launch_bump(ctx->st, 0, 1, ctx->stream);
    if (e) return fail(ctx, REWL_ECUDA, std::string("counter launch: ") + cudaGetErrorString((cudaError_t)e));
    ctx->launches += 1;
    return REWL_OK;
}

extern "C" rewl_status rewl_run(rewl_ctx *ctx, long n_sweeps)
{
    rewl_status s = check_usable(ctx);
    if (s) return s;
    if (n_sweeps < 0) return fail(ctx, REWL_EINVAL, "n_sweeps < 0");
    if ((s = plan(ctx))) return s;
    return enqueue_sweeps(ctx, n_sweeps);
}

extern "C" rewl_status rewl_exchange(rewl_ctx *ctx)
{
    rewl_status s = check_usable(ctx);
    if (s) return s;
    return enqueue_exchange(ctx);
}

extern "C" rewl_status rewl_run_cycles(rewl_ctx *ctx, long n_cycles, long sweeps_per_cycle)
{
    rewl_status s = check_usable(ctx);
    if (s) return s;
    if (n_cycles < 0 || sweeps_per_cycle < 1) return fail(ctx, REWL_EINVAL, "n_cycles < 0 or sweeps_per_cycle < 1");
    if ((s = plan(ctx))) return s;
    if (ctx->graph_sweeps != sweeps_per_cycle) {
        if (ctx->graph) {
            cudaGraphExecDestroy(ctx->graph);
            ctx->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        const long before = ctx->launches;
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        rewl_status a = enqueue_sweeps(ctx, sweeps_per_cycle);
        rewl_status b = a ? a : enqueue_exchange(ctx);
        cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
        if (b) return b;
        if (ce != cudaSuccess) return fail(ctx, REWL_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        ctx->graph_launches = ctx->launches - before;
        ctx->launches = before;
        cudaError_t ie = cudaGraphInstantiate(&ctx->graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return fail(ctx, REWL_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
        ctx->graph_sweeps = sweeps_per_cycle;
    }
    for (long c = 0; c < n_cycles; ++c) {
        CK(cudaGraphLaunch(ctx->graph, ctx->stream));
        ctx->launches += ctx->graph_launches;
    }
    return REWL_OK;
}

static rewl_status sync_and_check(rewl_ctx *ctx)
{
    CK(cudaStreamSynchronize(ctx->stream));
    int herr = 0;
    CK(d2h(ctx, &herr, ctx->d_error, 4));
    if (herr & kErrRange) return fail(ctx, REWL_EDEVICE, "ln g left the FP64-exact range |ln g| < 2^21");
    if (herr) return fail(ctx, REWL_EDEVICE, "device error word " + std::to_string(herr));
    return REWL_OK;
}

extern "C" rewl_status rewl_run_to_convergence(rewl_ctx *ctx, long exchange_interval, long max_sweeps,
                                               long poll_cycles, int *converged)
{
    rewl_status s = check_usable(ctx);
    if (s) return s;
    if (exchange_interval < 1 || max_sweeps < 0 || poll_cycles < 1)
        return fail(ctx, REWL_EINVAL, "exchange_interval, poll_cycles must be >= 1, max_sweeps >= 0");
    if (converged) *converged = 0;
    std::vector<uint8_t> conv(ctx->n_win);
    long done = 0;
    for (;;) {
        if ((s = sync_and_check(ctx))) return s;
        CK(d2h(ctx, conv.data(), ctx->d_conv, ctx->n_win));
        if (std::all_of(conv.begin(), conv.end(), [](uint8_t v) { return v != 0; })) {
            if (converged) *converged = 1;
            return REWL_OK;
        }
        if (done >= max_sweeps) return REWL_OK;
        long cycles = std::min(poll_cycles, std::max(1L, (max_sweeps - done) / exchange_interval));
        if ((s = rewl_run_cycles(ctx, cycles, exchange_interval))) return s;
        done += cycles * exchange_interval;
    }
}

// ---------------------------------------------------------------------------
// read-out
// ---------------------------------------------------------------------------
static rewl_status check_inst(rewl_ctx *ctx, int inst)
{
    if (!ctx) return REWL_EINVAL;
    if (inst < 0 || inst >= (int)ctx->inst.size()) return fail(ctx, REWL_EINVAL, "instance index out of range");
    if (ctx->failed) return REWL_ESTATE;
    return REWL_OK;
}

extern "C" rewl_status rewl_geometry(rewl_ctx *ctx, int inst, int *hh, int *m, int *B, int *w, int *lo,
                                     uint8_t *reach)
{
    if (!ctx || inst < 0 || inst >= (int)ctx->inst.size()) return REWL_EINVAL;
    const HostInst &h = ctx->inst[inst];
    if (hh) *hh = h.dev.h;
    if (m) *m = h.dev.m;
    if (B) *B = h.dev.B;
    if (w) *w = h.dev.w;
    if (lo) std::copy(h.lo.begin(), h.lo.end(), lo);
    if (reach) std::copy(h.reach.begin(), h.reach.end(), reach);
    return REWL_OK;
}

extern "C" rewl_status rewl_window_widths(rewl_ctx *ctx, int inst, int32_t *ww)
{
    if (!ctx || !ww || inst < 0 || inst >= (int)ctx->inst.size()) return REWL_EINVAL;
    const HostInst &h = ctx->inst[inst];
    std::copy(h.ww.begin(), h.ww.end(), ww);
    return REWL_OK;
}

template <class T>
static cudaError_t dget(rewl_ctx *ctx, std::vector<T> &v, const T *d, size_t n)
{
    v.resize(n);
    if (n == 0) return cudaSuccess;
    return d2h(ctx, v.data(), d, n * sizeof(T));
}

extern "C" rewl_status rewl_get_state(rewl_ctx *ctx, int inst, int8_t *spins, int64_t *E, int32_t *bin,
                                      double *ln_g, uint32_t *H, int32_t *stage, uint8_t *conv,
                                      uint8_t *latch, int64_t *replica)
{
    rewl_status s = check_inst(ctx, inst);
    if (s) return s;
    if ((s = sync_and_check(ctx))) return s;
    const InstDev &I = ctx->inst[inst].dev;
    const int nw = I.h * I.m;
    std::vector<int32_t> cfg, e, b, rep;
    CK(dget(ctx, cfg, ctx->d_cfg + I.slot0, nw));
    if (spins) {
        std::vector<uint32_t> lat;
        CK(dget(ctx, lat, ctx->d_lat + I.lat_off, (size_t)nw * I.lat_words));
        for (int k = 0; k < nw; ++k) {
            const uint32_t *l = lat.data() + (size_t)cfg[k] * I.lat_words;
            for (int y = 0; y < I.L; ++y)
                for (int x = 0; x < I.L; ++x) {
                    int v;
                    if (I.model == REWL_ISING) v = ((l[y * I.wpr + (x >> 5)] >> (x & 31)) & 1u) ? 1 : -1;
                    else v = reinterpret_cast<const uint8_t *>(l)[y * I.L + x];
                    spins[(size_t)k * I.N + y * I.L + x] = (int8_t)v;
                }
        }
    }
    if (E) {
        CK(dget(ctx, e, ctx->d_E + I.slot0, nw));
        for (int k = 0; k < nw; ++k) E[k] = e[k];
    }
    if (bin) CK(d2h(ctx, bin, ctx->d_bin + I.slot0, 4 * nw));
    if (ln_g) {
        std::vector<long long> u;
        CK(dget(ctx, u, ctx->d_lng + I.lng_off, (size_t)nw * I.w));
        for (size_t i = 0; i < u.size(); ++i) ln_g[i] = std::ldexp((double)u[i], -32);
    }
    if (H) {
        // converged windows count H; elsewhere H = (ln g - ln g at the stage
        // start) / ln f, exact in 2^-32 units with ln f = 2^(32 - stage)
        std::vector<long long> u, u0;
        std::vector<int32_t> sg;
        std::vector<uint8_t> cv;
        CK(dget(ctx, u, ctx->d_lng + I.lng_off, (size_t)nw * I.w));
        CK(dget(ctx, u0, ctx->d_lng0 + I.lng_off, (size_t)nw * I.w));
        CK(dget(ctx, sg, ctx->d_stage + I.win0, I.h));
        CK(dget(ctx, cv, ctx->d_conv + I.win0, I.h));
        CK(d2h(ctx, H, ctx->d_H + I.lng_off, 4 * (size_t)nw * I.w));
        for (int k = 0; k < nw; ++k) {
            const int win = k / I.m;
            if (cv[win]) continue;
            for (int bb = 0; bb < I.w; ++bb) {
                const size_t i = (size_t)k * I.w + bb;
                H[i] = (uint32_t)((u[i] - u0[i]) >> (32 - sg[win]));
            }
        }
    }
    if (stage) CK(d2h(ctx, stage, ctx->d_stage + I.win0, 4 * I.h));
    if (conv) CK(d2h(ctx, conv, ctx->d_conv + I.win0, I.h));
    if (latch) CK(d2h(ctx, latch, ctx->d_latch + I.slot0, nw));
    if (replica) {
        CK(dget(ctx, rep, ctx->d_replica + I.slot0, nw));
        for (int k = 0; k < nw; ++k) replica[k] = rep[k];
    }
    return REWL_OK;
}

extern "C" rewl_status rewl_get_counters(rewl_ctx *ctx, int inst, uint64_t *ex_prop, uint64_t *ex_acc,
                                         uint64_t *n_accepted, int64_t *conv_sweep)
{
    rewl_status s = check_inst(ctx, inst);
    if (s) return s;
    if ((s = sync_and_check(ctx))) return s;
    const InstDev &I = ctx->inst[inst].dev;
    if (ex_prop) CK(d2h(ctx, ex_prop, ctx->d_ex_prop + I.win0, 8 * I.h));
    if (ex_acc) CK(d2h(ctx, ex_acc, ctx->d_ex_acc + I.win0, 8 * I.h));
    if (n_accepted) CK(d2h(ctx, n_accepted, ctx->d_nacc + I.slot0, 8 * (size_t)I.h * I.m));
    if (conv_sweep) CK(d2h(ctx, conv_sweep, ctx->d_conv_sweep + I.win0, 8 * I.h));
    return REWL_OK;
}

extern "C" rewl_status rewl_get_stage_sweeps(rewl_ctx *ctx, int inst, int64_t *stage_sweep)
{
    rewl_status s = check_inst(ctx, inst);
    if (s) return s;
    if (!stage_sweep) return fail(ctx, REWL_EINVAL, "stage_sweep is NULL");
    if ((s = sync_and_check(ctx))) return s;
    const InstDev &I = ctx->inst[inst].dev;
    CK(d2h(ctx, stage_sweep, ctx->d_stage_sweep + (size_t)I.win0 * kMaxStages, 8 * (size_t)I.h * kMaxStages));
    return REWL_OK;
}

extern "C" rewl_status rewl_status_query(rewl_ctx *ctx, int inst, int *all_converged, double *ln_f_per_window,
                                         long *sweeps)
{
    rewl_status s = check_inst(ctx, inst);
    if (s) return s;
    if ((s = sync_and_check(ctx))) return s;
    if (all_converged) {
        std::vector<uint8_t> conv;
        CK(dget(ctx, conv, ctx->d_conv, ctx->n_win));
        *all_converged = std::all_of(conv.begin(), conv.end(), [](uint8_t v) { return v != 0; });
    }
    const InstDev &I = ctx->inst[inst].dev;
    if (ln_f_per_window) {
        std::vector<int32_t> st;
        std::vector<uint8_t> cv;
        CK(dget(ctx, st, ctx->d_stage + I.win0, I.h));
        CK(dget(ctx, cv, ctx->d_conv + I.win0, I.h));
        for (int i = 0; i < I.h; ++i) ln_f_per_window[i] = cv[i] ? 0.0 : std::ldexp(1.0, -st[i]);
    }
    if (sweeps) {
        ull c[2];
        CK(d2h(ctx, c, ctx->d_counters, 16));
        *sweeps = (long)c[0];
    }
    return REWL_OK;
}

// Sec. II B: join the pieces where their five-point inverse-temperature
// estimates agree best, above the previous join; normalise at the first
// realisable bin to ln_min.  pieces: h rows of w values (window i's bins
// lo[i] .. lo[i] + ww[i] - 1 first in its row).
static void join_geometry(int H, int w, int B, const int *lo, const int *ww, const uint8_t *reach, double dE,
                          double ln_min, const double *pieces, double *out)
{
    const int s = 1;
    for (int b = 0; b < B; ++b) out[b] = NAN;
    auto piece = [&](int i, int b) { return pieces[(size_t)i * w + (b - lo[i])]; };
    auto beta = [&](int i, int b) {
        return (piece(i, b - 2 * s) - 8.0 * piece(i, b - s) + 8.0 * piece(i, b + s) - piece(i, b + 2 * s)) /
               (12.0 * s * dE);
    };
    double shift = 0.0;
    int start = lo[0];
    for (int i = 0; i + 1 < H; ++i) {
        const int ov_lo = std::max(lo[i], lo[i + 1]);
        const int ov_hi = std::min(lo[i] + ww[i] - 1, lo[i + 1] + ww[i + 1] - 1);
        int best = -1;
        double best_d = 0.0;
        for (int b = std::max(ov_lo, start + 1); b <= ov_hi; ++b) {
            if (b - 2 * s < ov_lo || b + 2 * s > ov_hi) continue;
            bool ok = true;
            for (int d = -2; d <= 2; ++d) ok = ok && reach[b + d * s];
            if (!ok) continue;
            const double dd = std::fabs(beta(i, b) - beta(i + 1, b));
            if (best < 0 || dd < best_d) {
                best = b;
                best_d = dd;
            }
        }
        if (best < 0) {
            best = std::max(ov_lo, start + 1);
            while (best < ov_hi && !reach[best]) ++best;
        }
        for (int b = start; b < best; ++b) out[b] = piece(i, b) + shift;
        shift = piece(i, best) + shift - piece(i + 1, best);
        start = best;
    }
    for (int b = start; b < lo[H - 1] + ww[H - 1]; ++b) out[b] = piece(H - 1, b) + shift;
    int first = -1;
    for (int b = 0; b < B; ++b) {
        if (!reach[b]) out[b] = NAN;
        else if (first < 0) first = b;
    }
    const double off = ln_min - out[first];
    for (int b = 0; b < B; ++b) out[b] += off;
}

static void join_pieces(const HostInst &h, const std::vector<double> &pieces, std::vector<double> &out)
{
    const InstDev &I = h.dev;
    out.assign(I.B, NAN);
    join_geometry(I.h, I.w, I.B, h.lo.data(), h.ww.data(), h.reach.data(), (double)I.step,
                  std::log(I.model == REWL_ISING ? 2.0 : (double)I.q), pieces.data(), out.data());
}

extern "C" rewl_status rewl_join_pieces(int h, int w, int B, const int32_t *lo, const int32_t *ww,
                                        const uint8_t *reach, double bin_width, double ln_g_first,
                                        const double *pieces, double *ln_g)
{
    if (h < 1 || w < 5 || B < 1 || !lo || !ww || !reach || !pieces || !ln_g || !(bin_width > 0.0))
        return fail(nullptr, REWL_EINVAL, "rewl_join_pieces: bad argument");
    if (lo[0] != 0 || lo[h - 1] + ww[h - 1] != B)
        return fail(nullptr, REWL_EINVAL, "rewl_join_pieces: windows must cover bins 0 .. B - 1");
    for (int i = 0; i < h; ++i) {
        if (ww[i] < 5 || ww[i] > w || lo[i] < 0 || lo[i] + ww[i] > B)
            return fail(nullptr, REWL_EINVAL, "rewl_join_pieces: window " + std::to_string(i) + " out of range");
        if (i + 1 < h && (lo[i + 1] <= lo[i] || lo[i + 1] > lo[i] + ww[i] - 1 || lo[i + 1] + ww[i + 1] <= lo[i] + ww[i]))
            return fail(nullptr, REWL_EINVAL, "rewl_join_pieces: windows " + std::to_string(i) + " and " +
                                                  std::to_string(i + 1) + " must overlap with increasing ends");
    }
    bool any = false;
    for (int b = 0; b < B; ++b) any = any || reach[b];
    if (!any) return fail(nullptr, REWL_EINVAL, "rewl_join_pieces: no realisable bin");
    std::vector<int> vlo(lo, lo + h), vww(ww, ww + h);
    join_geometry(h, w, B, vlo.data(), vww.data(), reach, bin_width, ln_g_first, pieces, ln_g);
    return REWL_OK;
}

extern "C" rewl_status rewl_get_dos(rewl_ctx *ctx, int inst, double *ln_g, long cap, long *n_written,
                                    long *e_of_bin, int per_window)
{
    rewl_status s = check_inst(ctx, inst);
    if (s) return s;
    if (!ln_g) return fail(ctx, REWL_EINVAL, "ln_g is NULL");
    if ((s = sync_and_check(ctx))) return s;
    const HostInst &h = ctx->inst[inst];
    const InstDev &I = h.dev;
    const long need = per_window ? (long)I.h * I.w : (long)I.B;
    if (cap < need) return fail(ctx, REWL_EINVAL, "cap smaller than the result (" + std::to_string(need) + ")");
    std::vector<long long> u;
    CK(dget(ctx, u, ctx->d_lng + I.lng_off, (size_t)I.h * I.m * I.w));
    std::vector<double> pieces((size_t)I.h * I.w);
    for (int i = 0; i < I.h; ++i)
        for (int b = 0; b < I.w; ++b) {
            double acc = 0.0;
            for (int j = 0; j < I.m; ++j) acc += std::ldexp((double)u[((size_t)i * I.m + j) * I.w + b], -32);
            pieces[(size_t)i * I.w + b] = b < h.ww[i] ? acc / I.m : NAN;
        }
    if (per_window) {
        std::copy(pieces.begin(), pieces.end(), ln_g);
        if (e_of_bin)
            for (int i = 0; i < I.h; ++i)
                for (int b = 0; b < I.w; ++b) e_of_bin[(size_t)i * I.w + b] = I.e_min + (long)(h.lo[i] + b) * I.step;
    } else {
        std::vector<double> out;
        join_pieces(h, pieces, out);
        std::copy(out.begin(), out.end(), ln_g);
        if (e_of_bin)
            for (int b = 0; b < I.B; ++b) e_of_bin[b] = I.e_min + (long)b * I.step;
    }
    if (n_written) *n_written = need;
    return REWL_OK;
}

extern "C" rewl_status rewl_set_initial_lng(rewl_ctx *ctx, int inst, const double *ln_g0, double ln_f_start)
{
    rewl_status s = check_inst(ctx, inst);
    if (s) return s;
    if (!ln_g0) return fail(ctx, REWL_EINVAL, "ln_g0 is NULL");
    int k0 = -1;
    if (ln_f_start != 0.0) {
        int e = 0;
        const double mant = std::frexp(ln_f_start, &e);
        if (mant != 0.5 || e > 1 || e < -31) return fail(ctx, REWL_EINVAL, "ln_f_start must be 0 or 2^-k, 0 <= k <= 32");
        k0 = 1 - e;
    }
    if ((s = sync_and_check(ctx))) return s;
    const HostInst &h = ctx->inst[inst];
    const InstDev &I = h.dev;
    std::vector<long long> u((size_t)I.h * I.m * I.w);
    for (int i = 0; i < I.h; ++i)
        for (int b = 0; b < h.ww[i]; ++b) {
            double v = ln_g0[h.lo[i] + b];
            if (!std::isfinite(v)) v = 0.0;
            const double units = std::nearbyint(std::ldexp(v, 32));
            if (!(std::fabs(units) < std::ldexp(1.0, 53))) return fail(ctx, REWL_EINVAL, "ln_g0 outside |ln g| < 2^21");
            for (int j = 0; j < I.m; ++j) u[((size_t)i * I.m + j) * I.w + b] = (long long)units;
        }
    CK(h2d_sync(ctx, ctx->d_lng + I.lng_off, u.data(), 8 * u.size()));
    CK(h2d_sync(ctx, ctx->d_lng0 + I.lng_off, u.data(), 8 * u.size()));
    CK(cudaMemset(ctx->d_H + I.lng_off, 0, 4 * u.size()));
    CK(cudaMemset(ctx->d_latch + I.slot0, 0, (size_t)I.h * I.m));
    CK(cudaMemset(ctx->d_stage_sweep + (size_t)I.win0 * kMaxStages, 0xFF, 8 * (size_t)I.h * kMaxStages));
    std::vector<int32_t> st(I.h, k0 < 0 ? 0 : k0);
    std::vector<uint8_t> cv(I.h, k0 < 0 ? 2 : 0);     // 2: sampling with frozen weights, H counted
    CK(h2d_sync(ctx, ctx->d_stage + I.win0, st.data(), 4 * I.h));
    CK(h2d_sync(ctx, ctx->d_conv + I.win0, cv.data(), I.h));
    return REWL_OK;
}

extern "C" rewl_status rewl_warm_start(rewl_ctx *ctx, int inst, rewl_mlp *net, double ln_f_start)
{
    rewl_status s = check_inst(ctx, inst);
    if (s) return s;
    if (!net) return fail(ctx, REWL_EINVAL, "rewl_warm_start: network is NULL");
    int k0 = -1;
    if (ln_f_start != 0.0) {
        int e = 0;
        const double mant = std::frexp(ln_f_start, &e);
        if (mant != 0.5 || e > 1 || e < -31) return fail(ctx, REWL_EINVAL, "ln_f_start must be 0 or 2^-k, 0 <= k <= 32");
        k0 = 1 - e;
    }
    if ((s = sync_and_check(ctx))) return s;
    const InstDev &I = ctx->inst[inst].dev;
    std::string why;
    const int rc = mlp_warm_start(net, ctx->st, inst, I.h, I.w, k0, why);
    if (rc) return fail(ctx, (rewl_status)rc, "warm start: " + why);
    CK(cudaMemset(ctx->d_stage_sweep + (size_t)I.win0 * kMaxStages, 0xFF, 8 * (size_t)I.h * kMaxStages));
    return REWL_OK;
}

extern "C" rewl_status rewl_set_option(rewl_ctx *ctx, int option, long value)
{
    if (!ctx) return REWL_EINVAL;
    switch (option) {
        case REWL_OPT_CHECK_EVERY:
            if (value < 1) return fail(ctx, REWL_EINVAL, "check_every must be >= 1");
            ctx->check_every = value;
            break;
        case REWL_OPT_PRODUCER_WARPS:
            if (value < 0 || value > 4) return fail(ctx, REWL_EINVAL, "producer warps must be in 0..4");
            if (ctx->planned) return fail(ctx, REWL_ESTATE, "launch plan already fixed");
            ctx->force_producers = (int)value;
            break;
        case REWL_OPT_WINDOWS_PER_CTA:
            if (value < 0) return fail(ctx, REWL_EINVAL, "windows per block must be >= 0");
            if (ctx->planned) return fail(ctx, REWL_ESTATE, "launch plan already fixed");
            ctx->force_wpc = (int)value;
            break;
        case REWL_OPT_AUTOTUNE:
            if (value != 0 && value != 1) return fail(ctx, REWL_EINVAL, "autotune must be 0 (rule) or 1 (measure)");
            if (ctx->planned) return fail(ctx, REWL_ESTATE, "launch plan already fixed");
            ctx->tune_mode = (int)value;
            break;
        case REWL_OPT_MAX_SWEEPS_PER_LAUNCH:
            if (value < 1) return fail(ctx, REWL_EINVAL, "max sweeps per launch must be >= 1");
            ctx->max_sweeps_per_launch = value;
            break;
        case REWL_OPT_LNG_SHIFT:
            if (value < 1 || value > 20) return fail(ctx, REWL_EINVAL, "ln g shift exponent must be in 1..20");
            ctx->shift_exp = (int)value;
            break;
        case REWL_OPT_LATTICE_PLACEMENT:
            if (value < 0 || value > 2) return fail(ctx, REWL_EINVAL, "lattice placement must be 0, 1 or 2");
            if (ctx->planned) return fail(ctx, REWL_ESTATE, "launch plan already fixed");
            ctx->lattice_mode = (int)value;
            break;
        default:
            return fail(ctx, REWL_EINVAL, "unknown option");
    }
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
        ctx->graph_sweeps = -1;
    }
    return REWL_OK;
}

extern "C" long rewl_launch_count(const rewl_ctx *ctx) { return ctx ? ctx->launches : 0; }

extern "C" rewl_status rewl_transfer_bytes(const rewl_ctx *ctx, int64_t *h2d, int64_t *d2h)
{
    if (!ctx) return REWL_EINVAL;
    if (h2d) *h2d = ctx->bytes_h2d;
    if (d2h) *d2h = ctx->bytes_d2h;
    return REWL_OK;
}

extern "C" const char *rewl_last_error(const rewl_ctx *ctx)
{
    if (!ctx) return g_create_error.c_str();
    return ctx->err.c_str();
}

// ---------------------------------------------------------------------------
// checkpoint
// ---------------------------------------------------------------------------
static const char kMagic[8] = {'R', 'E', 'W', 'L', 'C', 'K', 'P', '4'};

template <class T>
static bool wr(FILE *f, const std::vector<T> &v)
{
    const uint64_t n = v.size();
    return fwrite(&n, 8, 1, f) == 1 && (n == 0 || fwrite(v.data(), sizeof(T), n, f) == n);
}
template <class T>
static bool rd(FILE *f, std::vector<T> &v)
{
    uint64_t n = 0;
    if (fread(&n, 8, 1, f) != 1) return false;
    v.resize(n);
    return n == 0 || fread(v.data(), sizeof(T), n, f) == n;
}

#define STATE_ARRAYS(X)                               \
    X(int32_t, d_stage, ctx->n_win)                   \
    X(uint8_t, d_conv, ctx->n_win)                    \
    X(int64_t, d_conv_sweep, ctx->n_win)              \
    X(ull, d_ex_prop, ctx->n_win)                     \
    X(ull, d_ex_acc, ctx->n_win)                      \
    X(int64_t, d_stage_sweep, (size_t)ctx->n_win * kMaxStages) \
    X(int32_t, d_cfg, ctx->n_slots)                   \
    X(int32_t, d_E, ctx->n_slots)                     \
    X(int32_t, d_bin, ctx->n_slots)                   \
    X(int32_t, d_replica, ctx->n_slots)               \
    X(ull, d_draw, ctx->n_slots)                      \
    X(ull, d_nacc, ctx->n_slots)                      \
    X(uint8_t, d_latch, ctx->n_slots)                 \
    X(long long, d_lng, (size_t)ctx->n_lng)           \
    X(long long, d_lng0, (size_t)ctx->n_lng)          \
    X(uint32_t, d_H, (size_t)ctx->n_lng)              \
    X(uint32_t, d_lat, (size_t)ctx->n_lat)            \
    X(ull, d_counters, 2)

extern "C" rewl_status rewl_save(rewl_ctx *ctx, const char *path)
{
    rewl_status s = check_usable(ctx);
    if (s) return s;
    if (!path) return fail(ctx, REWL_EINVAL, "path is NULL");
    if ((s = sync_and_check(ctx))) return s;
    FILE *f = fopen(path, "wb");
    if (!f) return fail(ctx, REWL_EINVAL, std::string("cannot open ") + path);
    bool ok = fwrite(kMagic, 8, 1, f) == 1;
    std::vector<rewl_instance> desc;
    for (auto &h : ctx->inst) desc.push_back(h.desc);
    ok = ok && wr(f, desc);
    std::vector<long> opts = {ctx->check_every};
    ok = ok && wr(f, opts);
    std::vector<int32_t> wlo, whi;                   // every window, bin by bin
    for (auto &h : ctx->inst)
        for (int i = 0; i < h.dev.h; ++i) {
            wlo.push_back(h.lo[i]);
            whi.push_back(h.lo[i] + h.ww[i] - 1);
        }
    ok = ok && wr(f, wlo) && wr(f, whi);
#define SAVE_ONE(T, field, n)                                     \
    if (ok) {                                                     \
        std::vector<T> v;                                         \
        if (dget(ctx, v, ctx->field, n) != cudaSuccess) ok = false;    \
        ok = ok && wr(f, v);                                      \
    }
    STATE_ARRAYS(SAVE_ONE)
#undef SAVE_ONE
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail(ctx, REWL_EINVAL, std::string("writing ") + path + " failed");
    return REWL_OK;
}

extern "C" rewl_status rewl_load(rewl_ctx **out, const char *path, void *cuda_stream)
{
    if (!out || !path) return fail(nullptr, REWL_EINVAL, "rewl_load: null argument");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(nullptr, REWL_EINVAL, std::string("cannot open ") + path);
    char mg[8];
    std::vector<rewl_instance> desc;
    std::vector<long> opts;
    std::vector<int32_t> wlo, whi;
    bool ok = fread(mg, 8, 1, f) == 1 && memcmp(mg, kMagic, 8) == 0 && rd(f, desc) && rd(f, opts) && !desc.empty() &&
              rd(f, wlo) && rd(f, whi) && wlo.size() == whi.size();
    if (ok) {
        size_t total = 0;
        for (auto &d : desc) total += d.n_windows > 0 ? (size_t)d.n_windows : 0;
        ok = total == wlo.size();
    }
    if (!ok) {
        fclose(f);
        return fail(nullptr, REWL_EINVAL, std::string(path) + " is not a REWL checkpoint");
    }
    rewl_status s = create_batch(out, desc.data(), (int)desc.size(), wlo.data(), whi.data(), cuda_stream);
    if (s) {
        fclose(f);
        return s;
    }
    rewl_ctx *ctx = *out;
    ctx->check_every = opts.empty() ? 1 : opts[0];
#define LOAD_ONE(T, field, n)                                                                           \
    if (ok) {                                                                                           \
        std::vector<T> v;                                                                               \
        ok = rd(f, v) && v.size() == (size_t)(n);                                                      \
        if (ok && h2d_sync(ctx, ctx->field, v.data(), sizeof(T) * v.size()) != cudaSuccess) \
            ok = false;                                                                                 \
    }
    STATE_ARRAYS(LOAD_ONE)
#undef LOAD_ONE
    fclose(f);
    if (!ok) return fail(ctx, REWL_EINVAL, std::string(path) + ": truncated or mismatched checkpoint");
    return REWL_OK;
}

// ---------------------------------------------------------------------------
// primitive checks
// ---------------------------------------------------------------------------
extern "C" rewl_status rewl_debug_lam(const uint32_t *k_dev, int64_t *out_dev, long n)
{
    rewl_ctx *ctx = nullptr;
    int e = launch_debug_lam(k_dev, out_dev, n, nullptr);
    if (e) return fail(nullptr, REWL_ECUDA, cudaGetErrorString((cudaError_t)e));
    CK(cudaDeviceSynchronize());
    return REWL_OK;
}

extern "C" rewl_status rewl_debug_philox(uint32_t key0, uint32_t key1, const uint32_t *ctr_dev, uint32_t *out_dev,
                                         long n)
{
    rewl_ctx *ctx = nullptr;
    int e = launch_debug_philox(key0, key1, ctr_dev, out_dev, n, nullptr);
    if (e) return fail(nullptr, REWL_ECUDA, cudaGetErrorString((cudaError_t)e));
    CK(cudaDeviceSynchronize());
    return REWL_OK;
}
