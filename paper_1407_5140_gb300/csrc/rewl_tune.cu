// rewl_tune.cu -- launch-shape choice for the sweep kernel: lanes per walker
// (G) and windows per thread block, per size class.  Never changes results:
// every random number is keyed by (instance, window, walker, draw index), and
// walkers of one window always share a block.
#include <algorithm>

#include "rewl_internal.h"

namespace rewl {

static const int kSMs = 152;             // GB300
static const int kSmemBudget = 110 * 1024;  // two blocks per SM
static const int kMaxThreads = 256;

// Lanes per walker: with few walkers per SM the per-walker dependency chain
// bounds throughput, so more lanes take over the state-independent work
// (Philox, thresholds); with many walkers one lane per walker issues fewest
// instructions per trial.
static int pick_lanes(int total_walkers, int model, int N, int m)
{
    const int apb = model == kIsing ? 2 : 1;
    int lanes = total_walkers <= kSMs * 32 ? 4 : (total_walkers <= kSMs * 96 ? 2 : 1);
    while (lanes > 1 && (N % (apb * lanes) != 0 || m * lanes > kMaxThreads)) lanes /= 2;
    return lanes;
}

int autotune_plan(rewl_ctx *ctx)
{
    const int nc = class_count(ctx);
    const int tot = total_walkers(ctx);
    for (int c = 0; c < nc; ++c) {
        int model, N, w, m, lw;
        class_shape(ctx, c, &model, &N, &w, &m, &lw);
        const int apb = model == kIsing ? 2 : 1;
        int lanes = forced_lanes(ctx) ? forced_lanes(ctx) : pick_lanes(tot, model, N, m);
        if (N % (apb * lanes) != 0 || m * lanes > kMaxThreads) return 1;
        const int per_win = sweep_smem_bytes(m, 1, w, lw);
        if (per_win > 227 * 1024) return 1;
        int wpc = forced_wpc(ctx);
        if (!wpc) {
            wpc = std::max(1, 32 / (m * lanes));
            while (wpc > 1 && (sweep_smem_bytes(wpc * m, wpc, w, lw) > kSmemBudget ||
                               wpc * m * lanes > kMaxThreads))
                --wpc;
        }
        if (sweep_smem_bytes(wpc * m, wpc, w, lw) > 227 * 1024 || wpc * m * lanes > kMaxThreads) return 1;
        plan_class(ctx, c, wpc, lanes);
    }
    return 0;
}

}  // namespace rewl
