// rewl_tune.cu -- launch-shape choice for the sweep kernel: windows per thread
// block (walkers per consumer warp) and producer warps per block, per size
// class.  A rule maps (walkers-per-block target, producer bias) to a shape;
// the host library measures a few targets and biases on a shadow copy of the
// batch and keeps the fastest (rewl_api.cu: measure_shapes).  Never changes
// results: every random number is keyed by (instance, window, walker, draw
// index), walkers of one window always share a block, and each walker's
// trials are resolved in draw order by one consumer lane.
#include <cuda_runtime.h>

#include <algorithm>

#include "rewl_internal.h"

namespace rewl {

static const int kSmemBudget = 110 * 1024;   // leaves room for two blocks per SM

// Streaming multiprocessors of the current device (152 on a GB300).
static int device_sms()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n < 1) {
        cudaGetLastError();
        return 1;
    }
    return n;
}

// Walkers per block: with few walkers per SM the per-walker dependency chain
// bounds throughput and small blocks spread walkers over all SMs; with many
// walkers, full consumer warps issue fewest instructions per trial.
static int pick_walkers(int total_walkers, int sms)
{
    if (total_walkers <= sms * 32) return 8;
    if (total_walkers <= sms * 96) return 16;
    return 32;
}

// Producer warps: Philox and threshold work per trial is ~1.5 (Ising) to ~2.5
// (Potts) times the consumer's per-trial work; one producer lane serves one
// Philox block per round: one warp per eight walkers (Ising), per six (Potts).
static int pick_producers(int model, int nw)
{
    const int p = model == kIsing ? (nw + 7) / 8 : (nw + 5) / 6;
    return std::max(1, std::min(4, p));
}

int block_shape(const rewl_ctx *ctx, int model, int N, int w, int m, int lw, int *wpc_out, int *producers_out)
{
    const int sms = device_sms();
    const int target = tune_target(ctx), bias = tune_producer_bias(ctx);
    auto producers = [&](int wpc) {
        return forced_producers(ctx) ? forced_producers(ctx)
                                     : std::max(1, std::min(4, pick_producers(model, wpc * m) + bias));
    };
    auto smem = [&](int wpc) { return sweep_smem_bytes(wpc * m, wpc, w, lw, producers(wpc), N); };
    if (m > 32 || sweep_smem_bytes(m, 1, w, lw, 1, N) > 227 * 1024) return 1;
    // shared memory per block: room for two blocks per SM, unless the whole
    // batch at this shape has no more blocks than SMs (then one block may
    // take all of it, so wide windows do not split a small batch into more
    // blocks than there are SMs)
    const long long tot = total_walkers(ctx);
    auto fits = [&](int wpc) {
        const long long blocks = (tot + (long long)wpc * m - 1) / ((long long)wpc * m);
        return smem(wpc) <= (blocks <= sms ? 227 * 1024 : kSmemBudget);
    };
    int wpc = forced_wpc(ctx);
    if (!wpc) {
        wpc = std::max(1, (target ? target : pick_walkers((int)tot, sms)) / m);
        while (wpc > 1 && (wpc * m > 32 || !fits(wpc))) --wpc;
    }
    if (wpc * m > 32 || smem(wpc) > 227 * 1024) return 1;
    *wpc_out = wpc;
    *producers_out = producers(wpc);
    return 0;
}

int autotune_plan(rewl_ctx *ctx)
{
    const int nc = class_count(ctx);
    for (int c = 0; c < nc; ++c) {
        int model, N, w, m, lw, wpc, producers;
        class_shape(ctx, c, &model, &N, &w, &m, &lw);
        if (block_shape(ctx, model, N, w, m, lw, &wpc, &producers)) return 1;
        plan_class(ctx, c, wpc, producers);
    }
    return 0;
}

}  // namespace rewl
