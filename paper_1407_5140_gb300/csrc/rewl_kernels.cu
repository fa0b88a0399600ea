// rewl_kernels.cu -- sm_103a kernels of the replica-exchange Wang-Landau path.
//
//  init_kernel      one thread per walker: start configuration, random walk into
//                   the walker's energy window (stream 1 of its Philox key).
//  sweep_kernel     one thread block per group of whole windows (at most 32
//                   walkers): producer warps prepare the state-independent part
//                   of every trial (Philox draws, sites, thresholds) a round
//                   ahead, and one consumer warp resolves each walker's trials
//                   in draw order, one lane per walker.  The block copies its
//                   walkers' lattices and ln g into shared memory, runs n sweeps
//                   of Wang-Landau trials (Sec. II A), and after every
//                   check_every sweeps tests flatness (H read off ln g and its
//                   value at the stage start; warp shuffles for the per-walker
//                   reductions) and merges windows whose m walkers are all flat.
//  exchange_kernel  one thread per proposed swap of a window pair (Eq. (1),
//                   Fig. 2); swaps the configuration indices of the two slots.
//  bump_kernel      advances the device-side sweep / exchange counters, so a
//                   captured graph of the cycle can be replayed.
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

#include <mutex>
#include <type_traits>

#include "rewl_device.cuh"
#include "rewl_internal.h"

namespace rewl {

// ---------------------------------------------------------------------------
// init
// ---------------------------------------------------------------------------
__device__ int full_energy(const InstDev &I, const uint32_t *lat)
{
    int E = 0;
    for (int y = 0; y < I.L; ++y)
        for (int x = 0; x < I.L; ++x) {
            const int xr = x == I.L - 1 ? 0 : x + 1, yd = y == I.L - 1 ? 0 : y + 1;
            if (I.model == kIsing) {
                const int s = (int)ising_bit(lat, I.wpr, y, x);
                const int a = (int)ising_bit(lat, I.wpr, y, xr), b = (int)ising_bit(lat, I.wpr, yd, x);
                E -= (s == a ? 1 : -1) + (s == b ? 1 : -1);
            } else {
                const int s = potts_get(lat, y * I.L + x);
                E -= (s == potts_get(lat, y * I.L + xr)) + (s == potts_get(lat, yd * I.L + x));
            }
        }
    return E;
}

__global__ void init_kernel(DevState st, int n_slots, const int32_t *slot_inst)
{
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= n_slots) return;
    const InstDev I = st.inst[slot_inst[slot]];
    const int local = slot - I.slot0;
    const int win = local / I.m, j = local % I.m;
    const int gwin = I.win0 + win;
    const int lo = st.lo[gwin], hi = lo + st.ww[gwin] - 1;
    const int L = I.L, N = I.N;
    uint32_t *lat = st.lat + I.lat_off + (long long)local * I.lat_words;
    st.cfg[slot] = local;
    st.replica[slot] = local;
    // start: ground state below the infinite-temperature mean energy, else the
    // two-colour checkerboard (maximum energy)
    const long long E_lo = I.e_min + (long long)lo * I.step;
    const bool below = I.model == kIsing ? (E_lo < 0) : ((long long)I.q * E_lo < -2LL * N);
    for (int i = 0; i < I.lat_words; ++i) lat[i] = 0u;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            const int odd = (x + y) & 1;
            if (I.model == kIsing) {
                const uint32_t up = below ? 1u : (odd ? 0u : 1u);
                lat[y * I.wpr + (x >> 5)] |= up << (x & 31);
            } else {
                potts_set(lat, y * L + x, below ? 0 : odd);
            }
        }
    int E = full_energy(I, lat);
    const uint32_t c2 = ((uint32_t)win << 16) | (uint32_t)j;
    auto bin_of = [&](int e) { return (int)((e - I.e_min) / I.step); };
    auto inside = [&](int e) {
        if (e < I.e_min || e > I.e_min + (long long)(I.B - 1) * I.step) return false;
        const int b = bin_of(e);
        return b >= lo && b <= hi;
    };
    unsigned long long blk = 0;
    while (!inside(E)) {
        if (blk >= (1ull << 28)) {
            atomicOr(st.error, kErrInit);
            break;
        }
        const u32x4 r = philox10((uint32_t)blk, (uint32_t)(blk >> 32), c2, 1u, I.key0, I.key1);
        ++blk;
        if (I.model == kIsing) {
            const uint32_t rs[2] = {r.x, r.z};
            for (int t = 0; t < 2 && !inside(E); ++t) {
                const Site s = site_of((int)scale_u32(rs[t], (uint32_t)N), L, I.magic_L);
                E += 4 * ising_flip_dbin(lat, I.wpr, s);
                ising_flip(lat, I.wpr, s);
            }
        } else {
            const int site = (int)scale_u32(r.x, (uint32_t)N);
            const Site s = site_of(site, L, I.magic_L);
            const int old = potts_get(lat, site);
            const int nv = (old + 1 + (int)scale_u32(r.y, (uint32_t)(I.q - 1))) % I.q;
            E += potts_dE(lat, L, s, old, nv);
            potts_set(lat, site, nv);
        }
    }
    st.E[slot] = E;
    st.bin[slot] = bin_of(E);
    st.draw[slot] = 0ull;
    st.latch[slot] = 0;
    st.n_acc[slot] = 0ull;
}

// ---------------------------------------------------------------------------
// sweeps
// ---------------------------------------------------------------------------
// Trials per producer round and walker (a round is one slot of the ring).
static constexpr int kR = 32;
// Guard bins on each side of a walker's ln g array: the consumer reads ln g of
// the bins b-4..b+4 speculatively before it knows the energy change.
static constexpr int kGuard = 4;

int sweep_smem_bytes(int n_walkers, int n_win, int w, int lat_words, int producers, int N)
{
    (void)producers;
    (void)N;
    long long b = 0;
    b += 2LL * n_walkers * kR * 48;                     // trial ring, 2 slots (48-byte records)
    b += (long long)n_walkers * (w + 2 * kGuard) * 8;   // ln g with guards
    b += (long long)n_walkers * 8;                      // Philox draw counters
    b += (long long)n_walkers * (lat_words | 1) * 4;    // lattices, odd word stride
    b += ((long long)n_win * w + 15) / 16 * 16;         // reach
    b += (long long)n_win * 20;                         // window state
    b += ((long long)n_walkers + 15) / 16 * 16;         // latch
    b += 2LL * n_walkers * 4;                           // near masks, 2 slots
    b += 8 + (long long)n_walkers * 8;                  // smallest ln g per walker (8-byte aligned)
    return (int)b;
}

struct SweepArgs {
    long n_sweeps, check_every;
    int shift_exp;   // a running window's ln g is lowered by 2^shift_exp once all of it has reached that
};

// Trials per Philox block: Ising 2 (site, u) pairs, Potts 1 (site, value, u).
template <int MODEL>
struct Apb {
    static constexpr int value = MODEL == kIsing ? 2 : 1;
};

// State-independent part of one trial, written by a producer warp into the
// ring: byte offsets (from the start of the block's shared memory) of the
// site's lattice word (Ising) or byte (Potts) and of its four neighbours'
// (left, right, up, down); `aux` holds the bit position of the site (Ising;
// the masks mx, ml, mr select site / up / down, left and right bits) or the
// proposal offset (Potts: new value = old + aux mod q).  `lam` is the
// acceptance threshold.  Trials whose site or a neighbour is the previous
// trial's site ("near") are marked in a per-round bit mask beside the ring.
struct __align__(16) Trial {
    uint32_t a_s, a_l, a_r, a_u, a_d, aux;
    long long lam;
    uint32_t mx, ml, mr, pad;   // Ising: bit masks of site (and up/down), left, right
};

static_assert(sizeof(Trial) == 48, "ring records are 48 bytes");

__device__ __forceinline__ bool site_near(int prev, int site, const Site &s, int L)
{
    return prev == site || prev == s.y * L + s.xl || prev == s.y * L + s.xr || prev == s.yu * L + s.x ||
           prev == s.yd * L + s.x;
}

// The APB trials of one Philox block; *first / *last receive the block's
// first and last sites, and the return value has bit k set when trial k > 0
// is near trial k - 1 (the caller decides for trial 0).
template <int MODEL>
__device__ __forceinline__ uint32_t make_trials(Trial *out, unsigned long long blk, uint32_t c2, const InstDev &I,
                                                uint32_t lat_off, int *first, int *last)
{
    int prev = -1;
    uint32_t near_bits = 0;
    const u32x4 r = philox10((uint32_t)blk, (uint32_t)(blk >> 32), c2, 0u, I.key0, I.key1);
    if (MODEL == kIsing) {
        const uint32_t rs[2] = {r.x, r.z}, ru[2] = {r.y, r.w};
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int site = (int)scale_u32(rs[k], (uint32_t)I.N);
            const Site s = site_of(site, I.L, I.magic_L);
            const uint32_t row = lat_off + 4u * (uint32_t)(s.y * I.wpr);
            const uint32_t hx = 4u * (uint32_t)(s.x >> 5);
            Trial t;
            t.a_s = row + hx;
            t.a_l = row + 4u * (uint32_t)(s.xl >> 5);
            t.a_r = row + 4u * (uint32_t)(s.xr >> 5);
            t.a_u = lat_off + 4u * (uint32_t)(s.yu * I.wpr) + hx;
            t.a_d = lat_off + 4u * (uint32_t)(s.yd * I.wpr) + hx;
            if (prev >= 0 && site_near(prev, site, s, I.L)) near_bits |= 1u << k;
            t.aux = (uint32_t)(s.x & 31);
            t.mx = 1u << (s.x & 31);
            t.ml = 1u << (s.xl & 31);
            t.mr = 1u << (s.xr & 31);
            t.pad = 0u;
            t.lam = lam_threshold(ru[k] >> 8);
            out[k] = t;
            if (k == 0) *first = site;
            prev = site;
        }
        *last = prev;
    } else {
        const int site = (int)scale_u32(r.x, (uint32_t)I.N);
        const Site s = site_of(site, I.L, I.magic_L);
        const uint32_t L = (uint32_t)I.L;
        Trial t;
        t.a_s = lat_off + (uint32_t)site;
        t.a_l = lat_off + (uint32_t)s.y * L + (uint32_t)s.xl;
        t.a_r = lat_off + (uint32_t)s.y * L + (uint32_t)s.xr;
        t.a_u = lat_off + (uint32_t)s.yu * L + (uint32_t)s.x;
        t.a_d = lat_off + (uint32_t)s.yd * L + (uint32_t)s.x;
        t.aux = 1u + scale_u32(r.y, (uint32_t)(I.q - 1));
        t.mx = t.ml = t.mr = t.pad = 0u;
        t.lam = lam_threshold(r.z >> 8);
        out[0] = t;
        *first = site;
        *last = site;
    }
    return near_bits;
}

// Lattice words (Ising) or values (Potts) a trial reads: site, left, right, up, down.
struct Nbr {
    uint32_t s, l, r, u, d;
};

template <int MODEL>
__device__ __forceinline__ Nbr load_nbr(const unsigned char *smem, const Trial &t)
{
    Nbr n;
    if (MODEL == kIsing) {
        n.s = *reinterpret_cast<const uint32_t *>(smem + t.a_s);
        n.l = *reinterpret_cast<const uint32_t *>(smem + t.a_l);
        n.r = *reinterpret_cast<const uint32_t *>(smem + t.a_r);
        n.u = *reinterpret_cast<const uint32_t *>(smem + t.a_u);
        n.d = *reinterpret_cast<const uint32_t *>(smem + t.a_d);
    } else {
        n.s = smem[t.a_s];
        n.l = smem[t.a_l];
        n.r = smem[t.a_r];
        n.u = smem[t.a_u];
        n.d = smem[t.a_d];
    }
    return n;
}

// Bin change of a trial from the lattice values it reads.  Ising: flipping
// s_i changes E by 2 s_i sum_j s_j = 8 - 4 (#neighbours unlike s_i), i.e.
// 2 - #unlike bins of 4; the three in-row bits (left, right, up) sit at
// distinct positions and are counted with one population count.  Potts
// (Eq. (2)): (#neighbours equal to the old value) - (#equal to the new value).
template <int MODEL>
__device__ __forceinline__ int bin_change(const Nbr &n, const Trial &t, int q)
{
    if (MODEL == kIsing) {
        const uint32_t S = (n.s & t.mx) ? 0xFFFFFFFFu : 0u;
        const uint32_t row3 = ((n.l ^ S) & t.ml) | ((n.r ^ S) & t.mr) | ((n.u ^ S) & t.mx);
        return 2 - __popc(row3) - __popc((n.d ^ S) & t.mx);
    } else {
        const int old = (int)n.s;
        int nv = old + (int)(t.aux & 0xFFFFu);
        nv -= nv >= q ? q : 0;
        const int a = (int)n.l, b = (int)n.r, c = (int)n.u, d = (int)n.d;
        return ((a == old) + (b == old) + (c == old) + (d == old)) - ((a == nv) + (b == nv) + (c == nv) + (d == nv));
    }
}

// Predicated stores and reductions without branches.
__device__ __forceinline__ void st_shared_u32_if(bool p, uint32_t addr, uint32_t v)
{
    asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q st.shared.u32 [%1], %2;\n}" ::"r"((uint32_t)p),
                 "r"(addr), "r"(v)
                 : "memory");
}

__device__ __forceinline__ void st_shared_u8_if(bool p, uint32_t addr, uint32_t v)
{
    asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q st.shared.u8 [%1], %2;\n}" ::"r"((uint32_t)p),
                 "r"(addr), "r"(v)
                 : "memory");
}

__device__ __forceinline__ void st_global_u32_if(bool p, unsigned char *ptr, uint32_t v)
{
    asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q st.global.u32 [%1], %2;\n}" ::"r"((uint32_t)p),
                 "l"(ptr), "r"(v)
                 : "memory");
}

__device__ __forceinline__ void st_global_u8_if(bool p, unsigned char *ptr, uint32_t v)
{
    asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q st.global.u8 [%1], %2;\n}" ::"r"((uint32_t)p),
                 "l"(ptr), "r"(v)
                 : "memory");
}

// Ask for the cache line at ptr to be brought into L2 (a hint: no value is
// read and nothing waits for it).
__device__ __forceinline__ void prefetch_l2(const unsigned char *ptr)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
}

__device__ __forceinline__ void st_shared_s64_if(bool p, uint32_t addr, long long v)
{
    asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q st.shared.s64 [%1], %2;\n}" ::"r"((uint32_t)p),
                 "r"(addr), "l"(v)
                 : "memory");
}

__device__ __forceinline__ void red_add_global_u32_if(bool p, uint32_t *ptr, uint32_t v)
{
    // no "memory" clobber: H is read only after a block-wide barrier, and
    // shared-memory loads stay free to move across the reduction
    asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q red.relaxed.gpu.global.add.u32 [%1], %2;\n}" ::"r"(
                     (uint32_t)p),
                 "l"(ptr), "r"(v));
}

__device__ __forceinline__ void named_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void named_arrive(int id, int nthreads)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

enum : int { kBarFull = 1, kBarEmpty = 3 };  // ids 1, 2 (full) and 3, 4 (empty); 0 is __syncthreads

// One thread block = n_win whole windows (nw = n_win * m <= 32 walkers).
// Warp 0 is the consumer: lane t resolves walker t's trials in order.  Warps
// 1..P are producers: they draw the Philox blocks and fill the ring with the
// state-independent parts of each trial, one round (kR trials per walker)
// ahead of the consumer, handing slots over with named barriers.  The
// consumer keeps the trial chain short: the next trial's lattice values are
// read one trial ahead, before the current trial's move is stored, and its
// bin change is computed from them, so the current trial only waits for one
// ln g load.  A trial whose site or a neighbour is the previous trial's site
// (marked by the producers) ends the unrolled loop; lanes whose previous
// trial moved read its values again there.  H needs no per-trial work while
// ln f > 0 (it is read off ln g and its value at the stage start); converged
// windows no longer count it, and sampling with frozen weights counts it in
// global memory with fire-and-forget reductions.
// GLAT: the lattices stay in global memory (large L, where a walker's lattice
// would crowd shared memory); the trial records then hold byte offsets from
// the start of the walker's lattice, and each consumer lane reads and writes
// its own walker's lattice there (a thread sees its own earlier stores, and no
// other thread touches that lattice during the launch).
template <int MODEL, bool GLAT>
__global__ void __launch_bounds__(160, 1) sweep_kernel(DevState st, const WorkItem *items, SweepArgs args)
{
    constexpr int APB = Apb<MODEL>::value;
    extern __shared__ __align__(16) unsigned char smem[];
    const WorkItem it = items[blockIdx.x];
    const InstDev I = st.inst[it.inst];
    // w: the instance's widest window (row stride of ln g, H in global
    // memory); wr: the widest window of this block (row length in shared memory)
    const int m = I.m, w = I.w, wr = it.wrow, n_win = it.n_win;
    const int nw = n_win * m;
    const int tid = threadIdx.x, nthreads = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    const bool consumer = warp == 0;
    const bool valid = consumer && lane < nw;
    const int tv = (consumer && lane < nw) ? lane : 0;
    const int lw = I.lat_words;
    // shared-memory words per walker's lattice: an odd stride spreads walkers
    // over banks; none when the lattices stay in global memory
    const int lwp = GLAT ? 0 : (lw | 1);
    const int wg = wr + 2 * kGuard;

    Trial *ring = reinterpret_cast<Trial *>(smem);
    long long *lng_s = reinterpret_cast<long long *>(ring + 2 * nw * kR);
    unsigned long long *draw_s = reinterpret_cast<unsigned long long *>(lng_s + (size_t)nw * wg);
    uint32_t *lat_s = reinterpret_cast<uint32_t *>(draw_s + nw);
    uint8_t *reach_s = reinterpret_cast<uint8_t *>(lat_s + (size_t)nw * lwp);
    int *wst_s = reinterpret_cast<int *>(reach_s + ((size_t)n_win * wr + 15) / 16 * 16);
    int *wstage_s = wst_s;
    int *wconv_s = wst_s + n_win;
    int *wmerge_s = wst_s + 2 * n_win;
    int *wgwin_s = wst_s + 3 * n_win;
    int *wwid_s = wst_s + 4 * n_win;        // bins of each window
    uint8_t *latch_s = reinterpret_cast<uint8_t *>(wst_s + 5 * n_win);
    // per slot and walker: bit a set when trial a of the round is near trial a - 1
    uint32_t *nearm_s = reinterpret_cast<uint32_t *>(latch_s + (nw + 15) / 16 * 16);
    // per walker: its smallest ln g over the realisable bins (flatness pass)
    long long *lmin_s = reinterpret_cast<long long *>(
        (reinterpret_cast<uintptr_t>(nearm_s + 2 * nw) + 7) & ~static_cast<uintptr_t>(7));

    const int slot_base = I.slot0 + it.win_begin * m;
    uint32_t *Hblk = st.H + I.lng_off + (long long)it.win_begin * m * w;   // this block's histograms
    long long *lng0blk = st.lng0 + I.lng_off + (long long)it.win_begin * m * w;
    // ---- load state into shared memory
    for (int i = tid; i < nw * wg; i += nthreads) {
        const int k = i / wg, bb = i - k * wg - kGuard;
        long long v = 0;
        if (bb >= 0 && bb < wr) v = st.lng[I.lng_off + (long long)(it.win_begin * m + k) * w + bb];
        lng_s[i] = v;
    }
    if (!GLAT)
        for (int i = tid; i < nw * lw; i += nthreads) {
            const int k = i / lw, x = i - k * lw;
            lat_s[k * lwp + x] = st.lat[I.lat_off + (long long)st.cfg[slot_base + k] * lw + x];
        }
    for (int i = tid; i < n_win * wr; i += nthreads) {
        const int wl = i / wr, bb = i - wl * wr;
        const int gw = I.win0 + it.win_begin + wl;
        reach_s[i] = bb < st.ww[gw] ? st.reach[I.reach_off + st.lo[gw] + bb] : (uint8_t)0;
    }
    for (int i = tid; i < n_win; i += nthreads) {
        const int gwin = I.win0 + it.win_begin + i;
        wgwin_s[i] = gwin;
        wwid_s[i] = st.ww[gwin];
        wstage_s[i] = st.stage[gwin];
        wconv_s[i] = st.conv[gwin];
        wmerge_s[i] = 0;
    }
    for (int i = tid; i < 2 * nw; i += nthreads) nearm_s[i] = 0u;
    for (int i = tid; i < nw; i += nthreads) {
        latch_s[i] = st.latch[slot_base + i];
        draw_s[i] = st.draw[slot_base + i];
    }
    __syncthreads();

    // consumer state (lane tv)
    const int wl_c = tv / m;
    const int lo = st.lo[I.win0 + it.win_begin + wl_c];
    const int w_c = st.ww[I.win0 + it.win_begin + wl_c];   // the lane's window width
    int b = st.bin[slot_base + tv];
    long long *lng = lng_s + (size_t)tv * wg + kGuard - lo;   // indexed by global bin
    uint32_t *H = Hblk + (size_t)tv * w - lo;                  // global, indexed by global bin
    const int q = I.q, N = I.N;
    const int rounds = (N + kR - 1) / kR;
    unsigned long long n_acc = 0;
    const uint32_t lat_base = (uint32_t)(reinterpret_cast<unsigned char *>(lat_s) - smem);
    const unsigned long long sweep0 = st.counters[0];

    for (long sw = 0; sw < args.n_sweeps; ++sw) {
        if (!consumer) {
            // ---------------- producers ----------------
            // producer warp pw fills the records of walkers [w0, w0 + cw): task
            // tk of a round is Philox block tk / cw of walker w0 + tk % cw, so
            // consecutive lanes write consecutive ring records (no bank
            // conflicts) and the block before a task's block is task tk - cw,
            // held by this warp in this pass or the previous one
            const int n_pw = nthreads / 32 - 1, pw = warp - 1;
            const int w0 = pw * nw / n_pw, cw = (pw + 1) * nw / n_pw - w0;
            const int src = lane >= cw ? lane - cw : lane + 32 - cw;
            for (int k = 0; k < rounds; ++k) {
                const int slot = k & 1;
                if (k >= 2) named_sync(kBarEmpty + slot, nthreads);
                const int cnt = min(kR, N - k * kR);
                const int nblk = cnt / APB;
                const int total = cw * nblk;
                int last_prev = -1;
                for (int base = 0; base < total; base += 32) {
                    const int task = base + lane;
                    const bool act = task < total;
                    const int tk = act ? task : total - 1;
                    const int bi = tk / cw, wk = w0 + (tk - bi * cw);
                    const int wlk = wk / m, jk = wk - wlk * m;
                    const uint32_t c2 = ((uint32_t)(it.win_begin + wlk) << 16) | (uint32_t)jk;
                    const unsigned long long blk = draw_s[wk] + (unsigned long long)(k * (kR / APB) + bi);
                    Trial tr[APB];
                    int first, last;
                    uint32_t nbits = make_trials<MODEL>(tr, blk, c2, I, GLAT ? 0u : lat_base + 4u * (uint32_t)(wk * lwp),
                                                        &first, &last);
                    // the block's first trial against the last trial of the
                    // walker's previous block (none for the round's first
                    // block: the consumer reads that trial's values afresh)
                    const int p_same = __shfl_sync(0xffffffffu, last, src);
                    const int p_prev = __shfl_sync(0xffffffffu, last_prev, src);
                    if (bi > 0) {
                        const Site fs = site_of(first, I.L, I.magic_L);
                        if (site_near(lane >= cw ? p_same : p_prev, first, fs, I.L)) nbits |= 1u;
                    }
                    if (act) {
                        // ring layout [slot][trial][walker]: the consumer lanes
                        // read consecutive records, free of bank conflicts
                        Trial *dst = ring + ((size_t)slot * kR + bi * APB) * nw + wk;
#pragma unroll
                        for (int i = 0; i < APB; ++i) dst[(size_t)i * nw] = tr[i];
                        if (nbits) atomicOr(nearm_s + slot * nw + wk, nbits << (bi * APB));
                    }
                    last_prev = last;
                }
                named_arrive(kBarFull + slot, nthreads);
            }
        } else {
            // ---------------- consumer ----------------
            // window state: 0 running; 1 converged (ln g frozen, no histogram);
            // 2 sampling with frozen weights (ln g frozen, H counted)
            const bool frozen = wconv_s[wl_c] != 0;
            const bool counting = wconv_s[wl_c] == 2;
            const long long lnf = frozen ? 0 : (1LL << (32 - wstage_s[wl_c]));
            long long cur = lng[b];
            uint32_t acc_count = 0;
            const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
            // shared address of ln g of global bin 0 of this walker (bins lo..hi valid)
            const uint32_t lng_sa = (uint32_t)__cvta_generic_to_shared(lng_s + (size_t)tv * wg + kGuard) - 8u * (uint32_t)lo;
            // the lane's lattice: trial offsets are from the block's shared
            // memory, or from the walker's lattice in global memory
            unsigned char *glat = GLAT ? reinterpret_cast<unsigned char *>(
                                             st.lat + I.lat_off + (long long)st.cfg[slot_base + tv] * lw)
                                       : nullptr;
            const unsigned char *lbase = GLAT ? glat : smem;
            // the rounds of one sweep; kCountH adds the H counting of
            // frozen-weight sampling, compiled out where the warp has none: a run
            // of trials that end in the same bin is added to H when the walker
            // leaves the bin (and at the end of the sweep), one trial later
            uint32_t run = 0, prun = 0;
            bool pend = false;
            uint32_t *Hpend = H;
            auto sweep_rounds = [&](auto count_h) {
                constexpr bool kCountH = decltype(count_h)::value;
                for (int k = 0; k < rounds; ++k) {
                    const int slot = k & 1;
                    named_sync(kBarFull + slot, nthreads);
                    const int cnt = min(kR, N - k * kR);
                    const Trial *rr = ring + (size_t)slot * kR * nw + tv;   // record a at rr[a * nw]
                    // trials near their predecessor in any lane end a run of
                    // the loop below; the mask is cleared for the slot's next use
                    uint32_t nm = 0u;
                    if (valid) {
                        nm = nearm_s[slot * nw + tv];
                        nearm_s[slot * nw + tv] = 0u;
                    }
                    const uint32_t wm = __reduce_or_sync(0xffffffffu, nm);
                    Trial t = rr[0];
                    Trial t1 = rr[cnt > 1 ? nw : 0];
                    const Nbr n0 = load_nbr<MODEL>(lbase, t);
                    int db = bin_change<MODEL>(n0, t, q);     // bin change of the current trial
                    uint32_t sv = n0.s;                        // its site word (Ising) / value (Potts)
                    bool acc_prev = false;
                    int a = 0;
                    for (;;) {
                    const uint32_t later = wm & (0xFFFFFFFEu << a);   // near trials after a
                    const int a_end = later ? __ffs(later) - 1 : cnt;
    #pragma unroll 3
                    for (; a < a_end; ++a) {
                        const Trial t2 = rr[(size_t)(a + 2 < cnt ? a + 2 : cnt - 1) * nw];
                        // lattices in global memory: start moving trial a+2's
                        // rows towards L2 now, two trials before they are read
                        if (GLAT) {
                            prefetch_l2(glat + t2.a_s);
                            prefetch_l2(glat + t2.a_u);
                            prefetch_l2(glat + t2.a_d);
                        }
                        // the previous trial's H flush, its operands long ready
                        if (kCountH) red_add_global_u32_if(pend, Hpend, prun);
                        // the next trial's lattice values, read before this trial's move
                        const Nbr nn = load_nbr<MODEL>(lbase, t1);
                        // this trial's move: Ising flips one bit of the site word,
                        // Potts writes the new value
                        uint32_t moved;
                        if (MODEL == kIsing) {
                            moved = sv ^ t.mx;
                        } else {
                            int nv = (int)sv + (int)(t.aux & 0xFFFFu);
                            nv -= nv >= q ? q : 0;
                            moved = (uint32_t)nv;
                        }
                        // accept iff ln g(E') < ln g(E) + lam, i.e. with min(1, g(E)/g(E'))
                        const int bn = b + db;
                        const bool inw = (unsigned)(bn - lo) < (unsigned)w_c;
                        const long long thr = cur + t.lam;
                        // ln g of the proposed bin (shared memory holds cur at b,
                        // and guard cells beyond the window's edges)
                        const long long v = lng[bn];
                        const bool acc = inw && (v < thr);
                        if (GLAT) {
                            if (MODEL == kIsing) st_global_u32_if(valid && acc, glat + t.a_s, moved);
                            else st_global_u8_if(valid && acc, glat + t.a_s, moved);
                        } else {
                            if (MODEL == kIsing) st_shared_u32_if(valid && acc, sbase + t.a_s, moved);
                            else st_shared_u8_if(valid && acc, sbase + t.a_s, moved);
                        }
                        // the next trial's bin change and site word from the values
                        // read before this move (the flag above catches the cases
                        // where this move changes them; an Ising site word shared
                        // with this trial's site gets the flipped bit here)
                        const int db_next = bin_change<MODEL>(nn, t1, q);
                        uint32_t sv_next = nn.s;
                        if (MODEL == kIsing) sv_next ^= (acc && t1.a_s == t.a_s) ? t.mx : 0u;
                        if (kCountH) {
                            const bool leave = acc && db != 0;
                            pend = valid && counting && leave;
                            Hpend = H + b;
                            prun = run;
                            run = leave ? 1u : run + 1u;
                        }
                        b = acc ? bn : b;
                        cur = (acc ? v : cur) + lnf;
                        acc_count += acc ? 1u : 0u;
                        st_shared_s64_if(valid, lng_sa + 8u * (uint32_t)b, cur);
                        acc_prev = acc;
                        db = db_next;
                        sv = sv_next;
                        t = t1;
                        t1 = t2;
                    }
                    if (a >= cnt) break;
                    // trial a is near trial a - 1 in some lane: where that trial
                    // moved, db and sv were taken before the move -- read again
                    if (acc_prev && ((nm >> a) & 1u)) {
                        const Nbr nf = load_nbr<MODEL>(lbase, t);
                        db = bin_change<MODEL>(nf, t, q);
                        sv = nf.s;
                    }
                    }
                    if (k + 2 < rounds) named_arrive(kBarEmpty + slot, nthreads);
                }
            };
            if (__any_sync(0xffffffffu, valid && counting)) sweep_rounds(std::true_type{});
            else sweep_rounds(std::false_type{});
            red_add_global_u32_if(pend, Hpend, prun);
            red_add_global_u32_if(valid && counting && run != 0u, H + b, run);
            n_acc += acc_count;
        }
        __syncthreads();
        if (tid < nw) draw_s[tid] += (unsigned long long)(N / APB);
        // ---- end of sweep: flatness, merge, ln f schedule
        const unsigned long long sweeps_done = sweep0 + (unsigned long long)sw + 1ull;
        if (sweeps_done % (unsigned long long)args.check_every == 0ull) {
            // flatness per walker: one warp per walker, lanes split the bins
            for (int wk = warp; wk < nw; wk += nthreads / 32) {
                const int wlk = wk / m;
                const long long *lk = lng_s + (size_t)wk * wg + kGuard;
                const long long *l0 = lng0blk + (size_t)wk * w;
                const int shift = 32 - wstage_s[wlk];   // ln f = 2^(32 - stage) units
                unsigned long long mn = ~0ull, sum = 0ull;
                long long amax = 0, lmin = LLONG_MAX;
                for (int bb = lane; bb < wwid_s[wlk]; bb += 32) {
                    const long long v = lk[bb];
                    const long long av = v < 0 ? -v : v;
                    amax = av > amax ? av : amax;
                    if (reach_s[wlk * wr + bb]) {
                        const unsigned long long hv = (unsigned long long)((v - __ldcg(l0 + bb)) >> shift);
                        mn = hv < mn ? hv : mn;
                        sum += hv;
                        lmin = v < lmin ? v : lmin;
                    }
                }
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned long long omn = __shfl_xor_sync(0xffffffffu, mn, o);
                    const unsigned long long osm = __shfl_xor_sync(0xffffffffu, sum, o);
                    const long long oam = __shfl_xor_sync(0xffffffffu, amax, o);
                    const long long olm = __shfl_xor_sync(0xffffffffu, lmin, o);
                    mn = omn < mn ? omn : mn;
                    sum += osm;
                    amax = oam > amax ? oam : amax;
                    lmin = olm < lmin ? olm : lmin;
                }
                if (lane == 0) {
                    lmin_s[wk] = lmin;
                    if (amax >= (1LL << 53)) atomicOr(st.error, kErrRange);
                    const int n_reach = st.n_reach[I.win0 + it.win_begin + wlk];
                    // Sec. II A: min H >= p <H>; Eq. (8): min H >= a / sqrt(ln f),
                    // ln f = 2^-stage, as sqrt(ldexp(a * a, stage)) in IEEE doubles
                    const bool flat = I.flat_rule == 1
                                          ? (double)mn >= sqrt(ldexp(I.p_flat * I.p_flat, wstage_s[wlk]))
                                          : (double)mn * (double)n_reach >= I.p_flat * (double)sum;
                    if (!wconv_s[wlk] && !latch_s[wk] && flat) latch_s[wk] = 1;
                }
            }
            __syncthreads();
            // bit 0: merge the window; bit 1: lower its ln g by 2^shift_exp.  ln g
            // of a window is defined up to a constant (pieces are joined by
            // differences, Sec. II B; acceptance and Eq. (1) use differences
            // within a window), so a running window whose walkers' ln g has
            // reached 2^shift_exp on every realisable bin is lowered by that
            // much (ln g and the stage-start copy alike, so H is unchanged):
            // on large lattices the first stages add far more than 2^21 per bin
            const long long lshift = 1LL << (32 + args.shift_exp);
            for (int i = tid; i < n_win; i += nthreads) {
                int all = !wconv_s[i];
                long long wmin = LLONG_MAX;
                for (int jj = 0; jj < m; ++jj) {
                    all = all && latch_s[i * m + jj];
                    wmin = lmin_s[i * m + jj] < wmin ? lmin_s[i * m + jj] : wmin;
                }
                const int lower = !wconv_s[i] && wmin >= lshift;
                wmerge_s[i] = all | (lower << 1);
            }
            __syncthreads();
            // merge: ln g <- mean over the window's walkers (nearest 2^-32, ties
            // to even); the next stage starts from it (lng0 <- ln g, H <- 0)
            for (int i = tid; i < n_win * wr; i += nthreads) {
                const int ww = i / wr, bb = i - ww * wr;
                if (!wmerge_s[ww] || bb >= wwid_s[ww]) continue;
                if ((wmerge_s[ww] & 2) && reach_s[ww * wr + bb])
                    for (int jj = 0; jj < m; ++jj) {
                        lng_s[(size_t)(ww * m + jj) * wg + kGuard + bb] -= lshift;
                        lng0blk[(size_t)(ww * m + jj) * w + bb] -= lshift;
                    }
                if (!(wmerge_s[ww] & 1)) continue;
                long long sacc = 0;
                for (int jj = 0; jj < m; ++jj) sacc += lng_s[(size_t)(ww * m + jj) * wg + kGuard + bb];
                const long long mean = div_round_even(sacc, m);
                for (int jj = 0; jj < m; ++jj) {
                    lng_s[(size_t)(ww * m + jj) * wg + kGuard + bb] = mean;
                    lng0blk[(size_t)(ww * m + jj) * w + bb] = mean;
                    Hblk[(size_t)(ww * m + jj) * w + bb] = 0u;
                }
            }
            __syncthreads();
            for (int i = tid; i < n_win; i += nthreads) {
                const int f = wmerge_s[i];
                wmerge_s[i] = 0;
                if (!(f & 1)) continue;
                for (int jj = 0; jj < m; ++jj) latch_s[i * m + jj] = 0;
                st.stage_sweep[(size_t)wgwin_s[i] * kMaxStages + wstage_s[i]] = (long long)sweeps_done;
                if (wstage_s[i] >= I.stage_final) {
                    wconv_s[i] = 1;
                    st.conv_sweep[wgwin_s[i]] = (long long)sweeps_done;
                } else {
                    wstage_s[i] += 1;
                }
            }
        }
        __syncthreads();
    }

    // ---- write back
    if (valid) {
        st.bin[slot_base + tv] = b;
        st.E[slot_base + tv] = (int)(I.e_min + (long long)b * I.step);
        st.n_acc[slot_base + tv] += n_acc;
    }
    for (int i = tid; i < nw * wr; i += nthreads) {
        const int k = i / wr, bb = i - k * wr;
        st.lng[I.lng_off + (long long)(it.win_begin * m + k) * w + bb] = lng_s[(size_t)k * wg + kGuard + bb];
    }
    if (!GLAT)
        for (int i = tid; i < nw * lw; i += nthreads) {
            const int k = i / lw, x = i - k * lw;
            st.lat[I.lat_off + (long long)st.cfg[slot_base + k] * lw + x] = lat_s[k * lwp + x];
        }
    for (int i = tid; i < n_win; i += nthreads) {
        st.stage[wgwin_s[i]] = wstage_s[i];
        st.conv[wgwin_s[i]] = (uint8_t)wconv_s[i];
    }
    for (int i = tid; i < nw; i += nthreads) {
        st.latch[slot_base + i] = latch_s[i];
        st.draw[slot_base + i] = draw_s[i];
    }
}

static const void *sweep_fn(int model, bool glat)
{
    if (model == kIsing) return glat ? (const void *)sweep_kernel<kIsing, true> : (const void *)sweep_kernel<kIsing, false>;
    return glat ? (const void *)sweep_kernel<kPotts, true> : (const void *)sweep_kernel<kPotts, false>;
}

int prepare_sweep(int model, bool glat, int smem)
{
    // the attribute belongs to the kernel, not to a context: never lower it
    // below what another live context already needs
    static int granted[4] = {0, 0, 0, 0};
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    const int k = (model & 1) * 2 + (glat ? 1 : 0);
    if (smem <= granted[k]) return 0;
    granted[k] = smem;
    // every launch of the kernel asks for the largest shared-memory carveout, so
    // launches of different size classes can share an SM
    const void *fn = sweep_fn(model, glat);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return (int)e;
}

int launch_sweeps(const DevState &st, const SweepLaunch &sl, long n_sweeps, long check_every, int shift_exp,
                  void *stream)
{
    SweepArgs a{n_sweeps, check_every, shift_exp};
    cudaStream_t s = (cudaStream_t)stream;
    if (sl.threads < 64 || sl.threads > 160 || sl.threads % 32 || sl.max_walkers > 32) return (int)cudaErrorInvalidValue;
    if (sl.model == kIsing) {
        if (sl.glat) sweep_kernel<kIsing, true><<<sl.n_items, sl.threads, sl.smem, s>>>(st, sl.items, a);
        else sweep_kernel<kIsing, false><<<sl.n_items, sl.threads, sl.smem, s>>>(st, sl.items, a);
    } else {
        if (sl.glat) sweep_kernel<kPotts, true><<<sl.n_items, sl.threads, sl.smem, s>>>(st, sl.items, a);
        else sweep_kernel<kPotts, false><<<sl.n_items, sl.threads, sl.smem, s>>>(st, sl.items, a);
    }
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// exchange
// ---------------------------------------------------------------------------
__global__ void exchange_kernel(DevState st, const ExTask *t0, int n0, const ExTask *t1, int n1)
{
    const unsigned long long t = st.counters[1];
    const ExTask *tasks = (t & 1ull) ? t1 : t0;
    const int n = (t & 1ull) ? n1 : n0;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const ExTask tk = tasks[id];
    const InstDev I = st.inst[tk.inst];
    const int m = I.m, w = I.w, i = tk.i, j = tk.j;
    const uint32_t tl = (uint32_t)t, th = (uint32_t)(t >> 32);
    const u32x4 rs = philox10(tl, th, ((uint32_t)i << 16) | 0xFFFFu, 2u, I.key0, I.key1);
    const int shift = (int)scale_u32(rs.x, (uint32_t)m);
    const u32x4 ru = philox10(tl, th, ((uint32_t)i << 16) | (uint32_t)j, 2u, I.key0, I.key1);
    const int a = I.slot0 + i * m + j;
    const int bslot = I.slot0 + (i + 1) * m + (j + shift) % m;
    const int gw_a = I.win0 + i, gw_b = gw_a + 1;
    atomicAdd(&st.ex_prop[gw_a], 1ull);
    const int lo_a = st.lo[gw_a], lo_b = st.lo[gw_b];
    const int bx = st.bin[a], by = st.bin[bslot];
    if (bx < lo_b || bx > lo_b + st.ww[gw_b] - 1 || by < lo_a || by > lo_a + st.ww[gw_a] - 1) return;
    const long long *ga = st.lng + I.lng_off + (long long)(i * m + j) * w;
    const long long *gb = st.lng + I.lng_off + (long long)((i + 1) * m + (j + shift) % m) * w;
    // -ln of the Eq. (1) ratio, in 2^-32 units
    const long long cost = (ga[by - lo_a] - ga[bx - lo_a]) + (gb[bx - lo_b] - gb[by - lo_b]);
    if (cost < lam_threshold(ru.x >> 8)) {
        int tmp = st.cfg[a]; st.cfg[a] = st.cfg[bslot]; st.cfg[bslot] = tmp;
        tmp = st.E[a]; st.E[a] = st.E[bslot]; st.E[bslot] = tmp;
        st.bin[a] = by; st.bin[bslot] = bx;
        tmp = st.replica[a]; st.replica[a] = st.replica[bslot]; st.replica[bslot] = tmp;
        atomicAdd(&st.ex_acc[gw_a], 1ull);
    }
}

__global__ void bump_kernel(unsigned long long *counters, unsigned long long sweeps,
                            unsigned long long exchanges)
{
    counters[0] += sweeps;
    counters[1] += exchanges;
}

int launch_init(const DevState &st, int n_slots, const int32_t *slot_inst, void *stream)
{
    const int bs = 64;
    init_kernel<<<(n_slots + bs - 1) / bs, bs, 0, (cudaStream_t)stream>>>(st, n_slots, slot_inst);
    return (int)cudaGetLastError();
}

int launch_exchange(const DevState &st, const ExTask *tasks0, int n0, const ExTask *tasks1, int n1,
                    void *stream)
{
    const int n = n0 > n1 ? n0 : n1;
    if (n == 0) return 0;
    const int bs = 128;
    exchange_kernel<<<(n + bs - 1) / bs, bs, 0, (cudaStream_t)stream>>>(st, tasks0, n0, tasks1, n1);
    return (int)cudaGetLastError();
}

int launch_bump(const DevState &st, long sweeps, long exchanges, void *stream)
{
    bump_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(st.counters, (unsigned long long)sweeps,
                                                    (unsigned long long)exchanges);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// primitive checks
// ---------------------------------------------------------------------------
__global__ void debug_lam_kernel(const uint32_t *k, int64_t *out, long n)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = lam_threshold(k[i]);
}

__global__ void debug_philox_kernel(uint32_t k0, uint32_t k1, const uint32_t *ctr, uint32_t *out, long n)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const u32x4 r = philox10(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], k0, k1);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

int launch_debug_lam(const uint32_t *k, int64_t *out, long n, void *stream)
{
    if (n <= 0) return 0;
    debug_lam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(k, out, n);
    return (int)cudaGetLastError();
}

int launch_debug_philox(uint32_t k0, uint32_t k1, const uint32_t *ctr, uint32_t *out, long n, void *stream)
{
    if (n <= 0) return 0;
    debug_philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(k0, k1, ctr, out, n);
    return (int)cudaGetLastError();
}

}  // namespace rewl
