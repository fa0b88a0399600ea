// rewl_internal.h -- layout of the device state shared by the host library
// (rewl_api.cu) and the kernels (rewl_kernels.cu).
//
// Device memory layout (all instances of a context concatenated):
//   per instance   InstDev                      (read-only in kernels)
//   per window     lo, n_reach, stage, conv, conv_sweep, ex_prop, ex_acc
//   per walker     cfg (index of the configuration buffer it holds), E, bin,
//                  draw (Philox block counter of the sweep stream), latch,
//                  n_acc, replica
//   per walker     ln g [w] int64 (units of 2^-32), H [w] uint32
//   per config     lattice: Ising bit-packed rows (bit = 1 <=> spin +1),
//                  Potts one byte per site; padded to whole 32-bit words
//   per instance   reach [B] bytes (1 = energy realisable)
//   context        counters: sweeps done, exchange phases done; error word
#pragma once
#include <stdint.h>

namespace rewl {

enum : int { kIsing = 0, kPotts = 1 };

// WL stages k = 0..32 (ln f = 2^-k) a window can pass through.
enum : int { kMaxStages = 33 };

// Error word bits raised by kernels (sticky, OR-ed).
enum : int {
    kErrRange = 1,       // |ln g| reached 2^21 (FP64-exact range left)
    kErrInit = 2,        // init walk did not reach the window within its bound
    kErrConfig = 4       // a work item did not match its launch configuration
};

struct InstDev {
    int32_t model, L, q, N;
    int32_t wpr;          // Ising: 32-bit words per lattice row
    int32_t lat_words;    // 32-bit words per configuration
    uint32_t magic_L;     // ceil(2^32 / L): y = umulhi(site, magic_L)
    int32_t step;         // energy units per bin
    int64_t e_min;
    int32_t B, h, m, w;
    int32_t win0;         // global index of window 0
    int32_t slot0;        // global index of walker 0 (walker = window * m + j)
    int32_t reach_off;    // offset of reach[] in the context's reach array
    int32_t stage_final;  // converge after the merge of this stage
    int64_t lng_off;      // element offset of walker 0's ln g / H
    int64_t lat_off;      // word offset of configuration 0
    uint32_t key0, key1;  // Philox key
    double p_flat;        // rule 0: p; rule 1: a
    int32_t flat_rule;    // 0: min H >= p <H>; 1: min H >= a / sqrt(ln f)
    int32_t pad1;
};

// One thread block of the sweep kernel: n_win consecutive windows of one
// instance; wrow = the widest of them (its walkers' ln g rows in shared memory).
struct WorkItem {
    int32_t inst, win_begin, n_win, wrow;
};

// One exchange proposal: walker j of window i of an instance (window pair i, i+1).
struct ExTask {
    int32_t inst, i, j, pad;
};

struct DevState {
    const InstDev *inst;
    // per window (global index)
    const int32_t *lo;
    const int32_t *ww;        // bins of the window (InstDev::w is the widest)
    const int32_t *n_reach;
    int32_t *stage;
    uint8_t *conv;
    int64_t *conv_sweep;
    unsigned long long *ex_prop, *ex_acc;
    // per window and WL stage (kMaxStages each): the sweep count at which the
    // stage ended with a merge (-1: not yet)
    long long *stage_sweep;
    // per walker slot (global index)
    int32_t *cfg;
    int32_t *E;
    int32_t *bin;
    unsigned long long *draw;
    uint8_t *latch;
    unsigned long long *n_acc;
    int32_t *replica;
    // per walker, per bin
    long long *lng;
    // ln g when the window's current stage began.  Every trial adds ln f to
    // ln g of the bin it ends in, so while ln f > 0 the stage's histogram is
    // H = (ln g - lng0) / ln f exactly; H below counts visits only in
    // converged windows (ln f = 0) and stays 0 elsewhere.
    long long *lng0;
    uint32_t *H;
    // configurations
    uint32_t *lat;
    // per instance bins
    const uint8_t *reach;
    // context counters: [0] sweeps done, [1] exchange phases done
    unsigned long long *counters;
    int *error;
};

// Host-side launch plumbing (rewl_kernels.cu).
struct SweepLaunch {
    const WorkItem *items;  // device array
    int n_items;
    int threads;            // per block: 32 * (1 consumer warp + producers)
    int producers;          // producer warps per block (1..4)
    int smem;               // dynamic shared memory bytes
    int max_walkers;        // walkers per block (n_win * m) upper bound
    int max_w;              // window width upper bound
    int max_lat_words;
    int max_win;            // windows per block upper bound
    int model;              // all items of one launch share the model
    int glat;               // 1: lattices stay in global memory (large L)
};

int launch_init(const DevState &st, int n_slots, const int32_t *slot_inst, void *stream);
int launch_sweeps(const DevState &st, const SweepLaunch &sl, long n_sweeps, long check_every, int shift_exp,
                  void *stream);
int launch_exchange(const DevState &st, const ExTask *tasks0, int n0, const ExTask *tasks1, int n1,
                    void *stream);
int launch_bump(const DevState &st, long sweeps, long exchanges, void *stream);
int sweep_smem_bytes(int n_walkers, int n_win, int w, int lat_words, int producers, int N);
int prepare_sweep(int model, bool glat, int smem);
int launch_debug_lam(const uint32_t *k, int64_t *out, long n, void *stream);
int launch_debug_philox(uint32_t k0, uint32_t k1, const uint32_t *ctr, uint32_t *out, long n,
                        void *stream);

}  // namespace rewl

// The learned warm start (rewl_mlp.cu): predict ln g of every window of an
// instance and install it in its walkers (k0 = starting stage, -1 = frozen).
#include <string>
struct rewl_mlp;
namespace rewl {
struct DevState;
int mlp_warm_start(rewl_mlp *net, const DevState &st, int inst, int h, int w, int k0, std::string &why);
}  // namespace rewl

// Planning hooks between the host library and the autotuner (rewl_tune.cu).
struct rewl_ctx;
namespace rewl {
int autotune_plan(rewl_ctx *ctx);
// Windows per block and producer warps for blocks of m-walker windows with
// ln g rows of w bins (the measured or rule target, shrunk to fit shared
// memory); 0 on success, 1 if not even one window fits.
int block_shape(const rewl_ctx *ctx, int model, int N, int w, int m, int lw, int *wpc, int *producers);
void plan_class(rewl_ctx *ctx, int c, int wpc, int producers);
int class_count(const rewl_ctx *ctx);
int class_walkers(const rewl_ctx *ctx, int c);
void class_shape(const rewl_ctx *ctx, int c, int *model, int *N, int *w, int *m, int *lat_words);
int total_walkers(const rewl_ctx *ctx);
int forced_producers(const rewl_ctx *ctx);
int forced_wpc(const rewl_ctx *ctx);
int tune_target(const rewl_ctx *ctx);          // walkers-per-block target (0: rule)
int tune_producer_bias(const rewl_ctx *ctx);   // added to the rule's producer warps
}  // namespace rewl
