// rewl_kernels.cu -- sm_103a kernels of the replica-exchange Wang-Landau path.
//
//  init_kernel      one thread per walker: start configuration, random walk into
//                   the walker's energy window (stream 1 of its Philox key).
//  sweep_kernel     one thread block per group of whole windows; each walker is
//                   served by G lanes of a warp.  The block copies its walkers'
//                   lattices, ln g and H into shared memory, runs n sweeps of
//                   Wang-Landau trials (Sec. II A), and after every check_every
//                   sweeps tests flatness and merges windows whose m walkers are
//                   all flat (warp shuffles for the per-walker reductions).
//  exchange_kernel  one thread per proposed swap of a window pair (Eq. (1),
//                   Fig. 2); swaps the configuration indices of the two slots.
//  bump_kernel      advances the device-side sweep / exchange counters, so a
//                   captured graph of the cycle can be replayed.
#include <cuda_runtime.h>
#include <stdint.h>

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
    const int lo = st.lo[gwin], hi = lo + I.w - 1;
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
int sweep_smem_bytes(int n_walkers, int n_win, int w, int lat_words)
{
    long long b = 0;
    b += (long long)n_walkers * w * 8;             // ln g
    b += (long long)n_walkers * w * 4;             // H
    b += (long long)n_walkers * lat_words * 4;     // lattices
    b += ((long long)n_win * w + 15) / 16 * 16;    // reach
    b += (long long)n_win * 16;                    // window state
    b += ((long long)n_walkers + 15) / 16 * 16;    // latch
    return (int)b;
}

struct SweepArgs {
    long n_sweeps, check_every;
};

// Trials per Philox block: Ising 2 (site, u) pairs, Potts 1 (site, value, u).
template <int MODEL>
struct Apb {
    static constexpr int value = MODEL == kIsing ? 2 : 1;
};

template <int MODEL, int G>
__global__ void __launch_bounds__(256) sweep_kernel(DevState st, const WorkItem *items, SweepArgs args)
{
    constexpr int APB = Apb<MODEL>::value;
    constexpr int A = APB * G;                      // trials per round and walker
    extern __shared__ __align__(16) unsigned char smem[];
    const WorkItem it = items[blockIdx.x];
    const InstDev I = st.inst[it.inst];
    const int m = I.m, w = I.w, n_win = it.n_win;
    const int nw = n_win * m;                       // walkers in this block
    const int tid = threadIdx.x;
    const int g = tid % G;                          // lane within the walker group
    const int t = tid / G;                          // walker within the block
    const bool valid = t < nw;
    const int tv = valid ? t : 0;                   // padding lanes shadow walker 0
    const int lw = I.lat_words;

    long long *lng_s = reinterpret_cast<long long *>(smem);
    uint32_t *H_s = reinterpret_cast<uint32_t *>(lng_s + (size_t)nw * w);
    uint32_t *lat_s = H_s + (size_t)nw * w;
    uint8_t *reach_s = reinterpret_cast<uint8_t *>(lat_s + (size_t)nw * lw);
    int *wst_s = reinterpret_cast<int *>(reach_s + ((size_t)n_win * w + 15) / 16 * 16);
    int *wstage_s = wst_s;                          // [n_win]
    int *wconv_s = wst_s + n_win;                   // [n_win]
    int *wmerge_s = wst_s + 2 * n_win;              // [n_win]
    int *wgwin_s = wst_s + 3 * n_win;               // [n_win]
    uint8_t *latch_s = reinterpret_cast<uint8_t *>(wst_s + 4 * n_win);

    const int slot_base = I.slot0 + it.win_begin * m;
    // ---- load state into shared memory
    for (int i = tid; i < nw * w; i += blockDim.x) {
        const int k = i / w, b = i - k * w;
        const long long off = I.lng_off + (long long)(it.win_begin * m + k) * w + b;
        lng_s[i] = st.lng[off];
        H_s[i] = st.H[off];
    }
    for (int i = tid; i < nw * lw; i += blockDim.x) {
        const int k = i / lw, x = i - k * lw;
        const int c = st.cfg[slot_base + k];
        lat_s[i] = st.lat[I.lat_off + (long long)c * lw + x];
    }
    for (int i = tid; i < n_win * w; i += blockDim.x) {
        const int wl = i / w, b = i - wl * w;
        const int gwin = I.win0 + it.win_begin + wl;
        reach_s[i] = st.reach[I.reach_off + st.lo[gwin] + b];
    }
    for (int i = tid; i < n_win; i += blockDim.x) {
        const int gwin = I.win0 + it.win_begin + i;
        wgwin_s[i] = gwin;
        wstage_s[i] = st.stage[gwin];
        wconv_s[i] = st.conv[gwin];
        wmerge_s[i] = 0;
    }
    for (int i = tid; i < nw; i += blockDim.x) latch_s[i] = st.latch[slot_base + i];
    __syncthreads();

    const int wl = tv / m, j = tv - wl * m;          // window within block, walker within window
    const int slot = slot_base + tv;
    const int lo = st.lo[I.win0 + it.win_begin + wl];
    const int hi = lo + w - 1;
    int b = st.bin[slot];
    int E = st.E[slot];
    unsigned long long draw = st.draw[slot];
    unsigned long long n_acc = 0;
    long long *lng = lng_s + (size_t)tv * w - lo;     // indexed by global bin
    uint32_t *H = H_s + (size_t)tv * w - lo;
    uint32_t *lat = lat_s + (size_t)tv * lw;
    const uint32_t c2 = ((uint32_t)(it.win_begin + wl) << 16) | (uint32_t)j;
    const int L = I.L, N = I.N, wpr = I.wpr, q = I.q;
    const bool leader = (g == 0) && valid;
    const unsigned long long sweep0 = st.counters[0];
    const int rounds = N / A;                        // N is a multiple of A (checked on the host)

    for (long sw = 0; sw < args.n_sweeps; ++sw) {
        const bool frozen = wconv_s[wl] != 0;
        const long long lnf = frozen ? 0 : (1LL << (32 - wstage_s[wl]));
        for (int rd = 0; rd < rounds; ++rd) {
            // ---- every lane: one Philox block and its state-independent parts
            const unsigned long long blk = draw + (unsigned long long)(rd * G + g);
            const u32x4 r = philox10((uint32_t)blk, (uint32_t)(blk >> 32), c2, 0u, I.key0, I.key1);
            int my_site[APB];
            int my_prop[APB];
            long long my_lam[APB];
            if (MODEL == kIsing) {
                my_site[0] = (int)scale_u32(r.x, (uint32_t)N);
                my_lam[0] = lam_threshold(r.y >> 8);
                my_site[APB - 1] = (int)scale_u32(r.z, (uint32_t)N);
                my_lam[APB - 1] = lam_threshold(r.w >> 8);
                my_prop[0] = my_prop[APB - 1] = 0;
            } else {
                my_site[0] = (int)scale_u32(r.x, (uint32_t)N);
                my_prop[0] = 1 + (int)scale_u32(r.y, (uint32_t)(q - 1));
                my_lam[0] = lam_threshold(r.z >> 8);
            }
            // ---- gather the group's A trials into the leader (warp-wide)
            int site_a[A];
            int prop_a[A];
            long long lam_a[A];
#pragma unroll
            for (int a = 0; a < A; ++a) {
                const int src_lane = a / APB;
                const int which = a % APB;
                if (G == 1) {
                    site_a[a] = my_site[which];
                    prop_a[a] = my_prop[which];
                    lam_a[a] = my_lam[which];
                } else {
                    const int lane0 = (threadIdx.x & 31) - g;
                    site_a[a] = __shfl_sync(0xffffffffu, my_site[which], lane0 + src_lane);
                    prop_a[a] = __shfl_sync(0xffffffffu, my_prop[which], lane0 + src_lane);
                    lam_a[a] = __shfl_sync(0xffffffffu, my_lam[which], lane0 + src_lane);
                }
            }
            // ---- the leader resolves the trials in order (Sec. II A)
            if (leader) {
#pragma unroll
                for (int a = 0; a < A; ++a) {
                    const int site = site_a[a];
                    const Site s = site_of(site, L, I.magic_L);
                    int db, nv = 0;
                    if (MODEL == kIsing) {
                        db = ising_flip_dbin(lat, wpr, s);
                    } else {
                        const int old = potts_get(lat, site);
                        nv = old + prop_a[a];
                        nv = nv >= q ? nv - q : nv;
                        db = potts_dE(lat, L, s, old, nv);
                    }
                    const int bn = b + db;
                    bool acc = false;
                    if (bn >= lo && bn <= hi) acc = (lng[bn] - lng[b]) < lam_a[a];
                    if (acc) {
                        if (MODEL == kIsing) ising_flip(lat, wpr, s);
                        else potts_set(lat, site, nv);
                        b = bn;
                        E += db * I.step;
                        ++n_acc;
                    }
                    if (!frozen) lng[b] += lnf;
                    H[b] += 1u;
                }
            }
        }
        draw += (unsigned long long)rounds * G;
        __syncthreads();
        // ---- end of sweep: flatness, merge, ln f schedule
        const unsigned long long sweeps_done = sweep0 + (unsigned long long)sw + 1ull;
        if (sweeps_done % (unsigned long long)args.check_every == 0ull) {
            // flatness per walker: G lanes split the bins, shuffles combine
            unsigned long long mn = ~0ull, sum = 0ull;
            long long amax = 0;
            const bool test = valid && !frozen && !latch_s[tv];
            for (int bb = lo + g; bb <= hi; bb += G) {
                const long long v = lng[bb];
                const long long av = v < 0 ? -v : v;
                amax = av > amax ? av : amax;
                if (reach_s[wl * w + (bb - lo)]) {
                    const unsigned long long hv = H[bb];
                    mn = hv < mn ? hv : mn;
                    sum += hv;
                }
            }
#pragma unroll
            for (int o = 1; o < G; o <<= 1) {
                const unsigned long long omn = __shfl_xor_sync(0xffffffffu, mn, o);
                const unsigned long long osm = __shfl_xor_sync(0xffffffffu, sum, o);
                const long long oam = __shfl_xor_sync(0xffffffffu, amax, o);
                mn = omn < mn ? omn : mn;
                sum += osm;
                amax = oam > amax ? oam : amax;
            }
            if (valid && amax >= (1LL << 53)) atomicOr(st.error, kErrRange);
            if (leader && test) {
                const int n_reach = st.n_reach[I.win0 + it.win_begin + wl];
                if ((double)mn * (double)n_reach >= I.p_flat * (double)sum) latch_s[tv] = 1;
            }
            __syncthreads();
            for (int i = tid; i < n_win; i += blockDim.x) {
                int all = !wconv_s[i];
                for (int jj = 0; jj < m && all; ++jj) all = latch_s[i * m + jj];
                wmerge_s[i] = all;
            }
            __syncthreads();
            // merge: ln g <- mean over the window's walkers (nearest 2^-32, ties
            // to even), H <- 0
            for (int i = tid; i < n_win * w; i += blockDim.x) {
                const int ww = i / w, bb = i - ww * w;
                if (!wmerge_s[ww]) continue;
                long long s = 0;
                for (int jj = 0; jj < m; ++jj) s += lng_s[(size_t)(ww * m + jj) * w + bb];
                const long long mean = div_round_even(s, m);
                for (int jj = 0; jj < m; ++jj) {
                    lng_s[(size_t)(ww * m + jj) * w + bb] = mean;
                    H_s[(size_t)(ww * m + jj) * w + bb] = 0u;
                }
            }
            __syncthreads();
            for (int i = tid; i < n_win; i += blockDim.x) {
                if (!wmerge_s[i]) continue;
                for (int jj = 0; jj < m; ++jj) latch_s[i * m + jj] = 0;
                if (wstage_s[i] >= I.stage_final) {
                    wconv_s[i] = 1;
                    st.conv_sweep[wgwin_s[i]] = (long long)sweeps_done;
                } else {
                    wstage_s[i] += 1;
                }
                wmerge_s[i] = 0;
            }
            __syncthreads();
        }
    }

    // ---- write back
    if (leader) {
        st.bin[slot] = b;
        st.E[slot] = E;
        st.draw[slot] = draw;
        st.n_acc[slot] += n_acc;
    }
    __syncthreads();
    for (int i = tid; i < nw * w; i += blockDim.x) {
        const int k = i / w, bb = i - k * w;
        const long long off = I.lng_off + (long long)(it.win_begin * m + k) * w + bb;
        st.lng[off] = lng_s[i];
        st.H[off] = H_s[i];
    }
    for (int i = tid; i < nw * lw; i += blockDim.x) {
        const int k = i / lw, x = i - k * lw;
        const int c = st.cfg[slot_base + k];
        st.lat[I.lat_off + (long long)c * lw + x] = lat_s[i];
    }
    for (int i = tid; i < n_win; i += blockDim.x) {
        st.stage[wgwin_s[i]] = wstage_s[i];
        st.conv[wgwin_s[i]] = (uint8_t)wconv_s[i];
    }
    for (int i = tid; i < nw; i += blockDim.x) st.latch[slot_base + i] = latch_s[i];
}

template <int MODEL, int G>
static cudaError_t launch_sweep_t(const DevState &st, const SweepLaunch &sl, SweepArgs a,
                                  cudaStream_t s)
{
    sweep_kernel<MODEL, G><<<sl.n_items, sl.threads, sl.smem, s>>>(st, sl.items, a);
    return cudaGetLastError();
}

template <int MODEL, int G>
static cudaError_t prepare_t(int smem)
{
    return cudaFuncSetAttribute(sweep_kernel<MODEL, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

int prepare_sweep(int model, int lanes, int smem)
{
    cudaError_t e = cudaErrorInvalidValue;
    if (model == kIsing) {
        switch (lanes) {
            case 1: e = prepare_t<kIsing, 1>(smem); break;
            case 2: e = prepare_t<kIsing, 2>(smem); break;
            case 4: e = prepare_t<kIsing, 4>(smem); break;
            case 8: e = prepare_t<kIsing, 8>(smem); break;
        }
    } else {
        switch (lanes) {
            case 1: e = prepare_t<kPotts, 1>(smem); break;
            case 2: e = prepare_t<kPotts, 2>(smem); break;
            case 4: e = prepare_t<kPotts, 4>(smem); break;
            case 8: e = prepare_t<kPotts, 8>(smem); break;
        }
    }
    return (int)e;
}

int launch_sweeps(const DevState &st, const SweepLaunch &sl, long n_sweeps, long check_every, void *stream)
{
    SweepArgs a{n_sweeps, check_every};
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaErrorInvalidValue;
    if (sl.model == kIsing) {
        switch (sl.lanes) {
            case 1: e = launch_sweep_t<kIsing, 1>(st, sl, a, s); break;
            case 2: e = launch_sweep_t<kIsing, 2>(st, sl, a, s); break;
            case 4: e = launch_sweep_t<kIsing, 4>(st, sl, a, s); break;
            case 8: e = launch_sweep_t<kIsing, 8>(st, sl, a, s); break;
        }
    } else {
        switch (sl.lanes) {
            case 1: e = launch_sweep_t<kPotts, 1>(st, sl, a, s); break;
            case 2: e = launch_sweep_t<kPotts, 2>(st, sl, a, s); break;
            case 4: e = launch_sweep_t<kPotts, 4>(st, sl, a, s); break;
            case 8: e = launch_sweep_t<kPotts, 8>(st, sl, a, s); break;
        }
    }
    return (int)e;
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
    if (bx < lo_b || bx > lo_b + w - 1 || by < lo_a || by > lo_a + w - 1) return;
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
