// Device-wide exclusive scans and an LSD radix sort of (key, value) pairs.
//
// Scans are reduce-then-scan: per-block totals, one block scanning the totals,
// then per-block scans seeded with their offsets.  Inside a block the scan is
// a warp shuffle scan over per-thread sums.
//
// The radix sort processes 8 bits per pass.  A pass is (1) a per-block digit
// histogram, (2) an exclusive scan of the digit-major histogram table, (3) a
// stable scatter.  Stability inside a block comes from warp-level ranking:
// __match_any_sync groups the lanes holding the same digit, popc of the lower
// lanes of that group gives the lane's rank, and per-warp digit counts in
// shared memory order the warps; rounds inside a block keep a running count
// per digit.  Every pass is therefore stable, so an LSD sequence of passes
// sorts by the full key and keeps equal keys in input order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "dv_internal.cuh"

namespace dv {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive block scan of one value per thread; returns the block total via *total.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T x, T* total) {
    __shared__ T warp_sums[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = warp_incl_scan(x);
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = lane < SCAN_THREADS / 32 ? warp_sums[lane] : T(0);
        T wi = warp_incl_scan(w);
        if (lane < SCAN_THREADS / 32) warp_sums[lane] = wi - w;
        if (lane == SCAN_THREADS / 32 - 1) *total = wi;
    }
    __syncthreads();
    T r = incl - x + warp_sums[warp];
    __syncthreads();
    return r;
}

template <typename Tin, typename Tout>
__global__ void k_scan_reduce(const Tin* __restrict__ in, int64_t n, Tout* __restrict__ bsum) {
    pdl_wait();
    pdl_launch_dependents();
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    Tout s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < n) s += (Tout)in[base + i];
    __shared__ Tout tot;
    block_excl_scan<Tout>(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// single block: in-place exclusive scan of the block sums, writes the grand total
template <typename Tout>
__global__ void k_scan_top(Tout* __restrict__ bsum, int64_t nb, Tout* __restrict__ total) {
    pdl_wait();
    pdl_launch_dependents();
    __shared__ Tout carry_s;
    __shared__ Tout tot;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += SCAN_THREADS) {
        int64_t i = b0 + threadIdx.x;
        Tout x = i < nb ? bsum[i] : Tout(0);
        Tout e = block_excl_scan<Tout>(x, &tot);
        Tout c = carry_s;
        if (i < nb) bsum[i] = c + e;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = c + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry_s;
}

template <typename Tin, typename Tout>
__global__ void k_scan_down(const Tin* __restrict__ in, int64_t n, const Tout* __restrict__ bsum,
                            Tout* __restrict__ out) {
    pdl_wait();
    pdl_launch_dependents();
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    Tout v[SCAN_ITEMS];
    Tout s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = base + i < n ? (Tout)in[base + i] : Tout(0);
        s += v[i];
    }
    __shared__ Tout tot;
    Tout run = block_excl_scan<Tout>(s, &tot) + bsum[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

template <typename Tin, typename Tout>
cudaError_t scan_impl(const Tin* in, Tout* out, int64_t n, Tout* total_dev, Arena& ar, cudaStream_t s) {
    if (n <= 0) {
        if (total_dev) return cudaMemsetAsync(total_dev, 0, sizeof(Tout), s);
        return cudaSuccess;
    }
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    Tout* bsum = ar.alloc<Tout>((size_t)nb);
    if (!bsum) return ar.err;
    launch_pdl(k_scan_reduce<Tin, Tout>, dim3((unsigned)nb), dim3(SCAN_THREADS), s, in, n, bsum);
    count_launches(1);
    launch_pdl(k_scan_top<Tout>, dim3(1), dim3(SCAN_THREADS), s, bsum, nb, total_dev);
    count_launches(1);
    if (out) {
        launch_pdl(k_scan_down<Tin, Tout>, dim3((unsigned)nb), dim3(SCAN_THREADS), s, in, n, bsum, out);
        count_launches(1);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// radix sort
// ---------------------------------------------------------------------------

constexpr int RS_THREADS = 256;
constexpr int RS_MAX_ROUNDS = 16;  // keys per thread per pass, chosen per sort (see radix_impl)
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_RADIX = 256;

template <typename K>
__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const K* __restrict__ keys, int64_t n, int shift,
                                                            uint32_t mask, uint32_t* __restrict__ hist,
                                                            int64_t nblocks, int rounds) {
    pdl_wait();
    pdl_launch_dependents();
    __shared__ uint32_t h[RS_RADIX];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_THREADS * rounds;
#pragma unroll 4
    for (int r = 0; r < rounds; ++r) {
        int64_t i = base + (int64_t)r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & mask], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

template <typename K>
__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(const K* __restrict__ keys,
                                                               const uint32_t* __restrict__ vals, int64_t n,
                                                               int shift, uint32_t mask,
                                                               const uint32_t* __restrict__ offs, int64_t nblocks,
                                                               K* __restrict__ okeys, uint32_t* __restrict__ ovals,
                                                               int rounds) {
    pdl_wait();
    pdl_launch_dependents();
    __shared__ uint32_t run[RS_RADIX];       // next free slot per digit (global index)
    __shared__ uint32_t wcnt[RS_WARPS][RS_RADIX];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    run[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    for (int w = 0; w < RS_WARPS; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_THREADS * rounds;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < rounds; ++r) {
        int64_t i = base + (int64_t)r * RS_THREADS + threadIdx.x;
        bool ok = i < n;
        K key = ok ? keys[i] : K(0);
        uint32_t val = ok ? vals[i] : 0u;
        uint32_t d = ok ? ((uint32_t)(key >> shift) & mask) : 0xffffffffu;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt);
        bool leader = rank == 0;
        if (ok && leader) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (ok) {
            uint32_t before = 0;
            for (int w = 0; w < warp; ++w) before += wcnt[w][d];
            uint32_t pos = run[d] + before + (uint32_t)rank;
            okeys[pos] = key;
            ovals[pos] = val;
        }
        __syncthreads();
        uint32_t add = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            add += wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = 0;
        }
        run[threadIdx.x] += add;
        __syncthreads();
    }
}

template <typename K>
cudaError_t radix_impl(K*& keys, uint32_t*& vals, K* keys_alt, uint32_t* vals_alt, int64_t n, int n_bits, Arena& ar,
                       cudaStream_t s) {
    if (n <= 1 || n_bits <= 0) return cudaSuccess;
    // keys per block: as many as possible while still giving every SM two blocks
    int rounds = RS_MAX_ROUNDS;
    while (rounds > 1 && (n + (int64_t)RS_THREADS * rounds - 1) / ((int64_t)RS_THREADS * rounds) < 304) rounds >>= 1;
    const int64_t tile = (int64_t)RS_THREADS * rounds;
    int64_t nblocks = (n + tile - 1) / tile;
    uint32_t* hist = ar.alloc<uint32_t>((size_t)(nblocks * RS_RADIX));
    uint32_t* offs = ar.alloc<uint32_t>((size_t)(nblocks * RS_RADIX));
    if (!hist || !offs) return ar.err;
    K* src_k = keys;
    uint32_t* src_v = vals;
    K* dst_k = keys_alt;
    uint32_t* dst_v = vals_alt;
    for (int shift = 0; shift < n_bits; shift += 8) {
        int bits = n_bits - shift < 8 ? n_bits - shift : 8;
        uint32_t mask = (1u << bits) - 1u;
        launch_pdl(k_radix_hist<K>, dim3((unsigned)nblocks), dim3(RS_THREADS), s, src_k, n, shift, mask, hist, nblocks, rounds);
        count_launches(1);
        cudaError_t e = scan_impl<uint32_t, uint32_t>(hist, offs, nblocks * RS_RADIX, nullptr, ar, s);
        if (e != cudaSuccess) return e;
        launch_pdl(k_radix_scatter<K>, dim3((unsigned)nblocks), dim3(RS_THREADS), s, src_k, src_v, n, shift, mask, offs, nblocks, dst_k, dst_v, rounds);
        count_launches(1);
        K* tk = src_k;
        src_k = dst_k;
        dst_k = tk;
        uint32_t* tv = src_v;
        src_v = dst_v;
        dst_v = tv;
    }
    keys = src_k;
    vals = src_v;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// one-sweep radix sort: one kernel per 8-bit pass
//
// The global digit histogram of every pass is computed up front in one read of
// the keys.  A pass kernel then takes tiles in order from an atomic counter;
// each tile ranks its keys stably (as above), publishes its per-digit counts
// (flag AGG), looks back over its predecessors for its exclusive prefix -- an
// inclusive predecessor (flag INC) ends the walk -- publishes its inclusive
// count and scatters.  A tile only waits on tiles that took their index
// earlier, so every wait ends; each spin is still bounded, and a bound that
// runs out ends the tile's walk and sets the device's wait-error word, which
// the next render's size read-back reports as a timeout.
// ---------------------------------------------------------------------------

// this device's wait-error word: a pass whose look-back bound runs out sets it (as well as the
// call's own flag); the render's size read-back takes it and reports a timeout
__device__ uint32_t g_spin_error = 0u;

constexpr int OS_THREADS = 256;
constexpr int OS_MAX_PASSES = 8;
constexpr uint32_t OS_AGG = 1u << 30, OS_INC = 2u << 30, OS_VAL = (1u << 30) - 1u;
constexpr int OS_SPIN_LIMIT = 1 << 22;  // reads of a predecessor's status word before a pass gives up (~seconds)
constexpr int OS_LOOK = 32;  // predecessors read per look-back step (their loads are in flight together)

template <typename K>
__global__ void __launch_bounds__(OS_THREADS) k_os_hist(const K* __restrict__ keys, int64_t n, int n_passes,
                                                         int n_bits, uint32_t* __restrict__ ghist) {
    pdl_wait();
    pdl_launch_dependents();
    __shared__ uint32_t h[OS_MAX_PASSES][RS_RADIX];
    for (int p = 0; p < n_passes; ++p) h[p][threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const K k = keys[i];
        for (int p = 0; p < n_passes; ++p) {
            const int sh = 8 * p;
            const int bits = n_bits - sh < 8 ? n_bits - sh : 8;
            atomicAdd(&h[p][(uint32_t)(k >> sh) & ((1u << bits) - 1u)], 1u);
        }
    }
    __syncthreads();
    for (int p = 0; p < n_passes; ++p)
        if (h[p][threadIdx.x]) atomicAdd(&ghist[p * RS_RADIX + threadIdx.x], h[p][threadIdx.x]);
}

__device__ __forceinline__ uint32_t os_load(const uint32_t* p) { return *(const volatile uint32_t*)p; }

template <typename K, int ROUNDS>
__global__ void __launch_bounds__(OS_THREADS) k_os_pass(const K* __restrict__ keys, const uint32_t* __restrict__ vals,
                                                         int64_t n, int shift, uint32_t mask,
                                                         const uint32_t* __restrict__ hist,
                                                         uint32_t* __restrict__ status, uint32_t* __restrict__ counter,
                                                         uint32_t* __restrict__ err, K* __restrict__ okeys,
                                                         uint32_t* __restrict__ ovals, int spin_limit) {
    pdl_wait();
    pdl_launch_dependents();
    __shared__ uint32_t s_tile;
    __shared__ uint32_t run[RS_RADIX];
    __shared__ uint32_t wcnt[RS_WARPS][RS_RADIX];
    __shared__ uint32_t s_base[RS_RADIX];
    __shared__ uint32_t s_tot;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(counter, 1u);
    run[tid] = 0;
    for (int w = 0; w < RS_WARPS; ++w) wcnt[w][tid] = 0;
    // The tile's keys are loaded for tile blockIdx.x while the counter's answer is on its way (blocks
    // are almost always handed out in index order); a block that drew another tile loads again.
    K key[ROUNDS];
    uint32_t val[ROUNDS], dig[ROUNDS], rank[ROUNDS];
    auto load_tile = [&](uint32_t tl) {
        const int64_t b0 = (int64_t)tl * OS_THREADS * ROUNDS;
#pragma unroll
        for (int r = 0; r < ROUNDS; ++r) {
            const int64_t i = b0 + (int64_t)r * OS_THREADS + tid;
            const bool ok = i < n;
            key[r] = ok ? keys[i] : K(0);
            val[r] = ok ? vals[i] : 0u;
        }
    };
    load_tile(blockIdx.x);
    // first slot of every digit: exclusive scan of the pass's digit counts (every tile scans the 256
    // counts itself, which costs less than a launch)
    const uint32_t goff = block_excl_scan<uint32_t>(hist[tid], &s_tot);
    const uint32_t tile = s_tile;
    if (tile != blockIdx.x) load_tile(tile);  // block-uniform
    const int64_t base = (int64_t)tile * OS_THREADS * ROUNDS;
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const int64_t i = base + (int64_t)r * OS_THREADS + tid;
        dig[r] = i < n ? ((uint32_t)(key[r] >> shift) & mask) : 0xffffffffu;
    }
    // stable tile-local ranks, round by round
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const uint32_t d = dig[r];
        const bool ok = d != 0xffffffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rk = __popc(peers & lt);
        if (ok && rk == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (ok) {
            uint32_t before = 0;
            for (int w = 0; w < warp; ++w) before += wcnt[w][d];
            rank[r] = run[d] + before + (uint32_t)rk;
        }
        __syncthreads();
        uint32_t add = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            add += wcnt[w][tid];
            wcnt[w][tid] = 0;
        }
        run[tid] += add;
        __syncthreads();
    }
    // publish, look back, publish inclusive (thread tid owns digit tid)
    const uint32_t mine = run[tid];
    uint32_t* st = status + (size_t)tile * RS_RADIX + tid;
    if (tile == 0) {
        *(volatile uint32_t*)st = OS_INC | mine;
        s_base[tid] = goff;
    } else {
        *(volatile uint32_t*)st = OS_AGG | mine;
        // look back OS_LOOK predecessors at a time: their status words are loaded together, then
        // summed from the nearest one until an inclusive prefix; a word not yet published is
        // re-read (bounded)
        uint32_t excl = 0;
        int64_t t = (int64_t)tile - 1;
        bool fin = false;
        while (!fin && t >= 0) {
            uint32_t v[OS_LOOK];
#pragma unroll
            for (int i = 0; i < OS_LOOK; ++i) v[i] = t - i >= 0 ? os_load(status + (size_t)(t - i) * RS_RADIX + tid) : OS_INC;
#pragma unroll
            for (int i = 0; i < OS_LOOK; ++i) {
                if (fin) break;
                if (t - i < 0) {
                    fin = true;
                    break;
                }
                const uint32_t* sp = status + (size_t)(t - i) * RS_RADIX + tid;
                int spins = 0;
                while ((v[i] & ~OS_VAL) == 0 && ++spins < spin_limit) v[i] = os_load(sp);
                if ((v[i] & ~OS_VAL) == 0) {
                    atomicOr(err, 1u);
                    atomicOr(&g_spin_error, 1u);
                    fin = true;
                    break;
                }
                excl += v[i] & OS_VAL;
                if (v[i] & OS_INC) fin = true;
            }
            t -= OS_LOOK;
        }
        // (no fence: readers take nothing from this tile but the word itself)
        *(volatile uint32_t*)st = OS_INC | ((excl + mine) & OS_VAL);
        s_base[tid] = goff + excl;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const int64_t i = base + (int64_t)r * OS_THREADS + tid;
        if (i < n) {
            int64_t pos = (int64_t)s_base[dig[r]] + rank[r];
            pos = pos < n ? pos : n - 1;  // only a timed-out look-back can leave the range
            okeys[pos] = key[r];
            ovals[pos] = val[r];
        }
    }
}

template <typename K, int ROUNDS>
cudaError_t onesweep_impl(K*& keys, uint32_t*& vals, K* keys_alt, uint32_t* vals_alt, int64_t n, int n_bits,
                          uint32_t* call_err, int n_sm, Arena& ar, cudaStream_t s) {
    const int passes = (n_bits + 7) / 8;
    const int64_t tile = (int64_t)OS_THREADS * ROUNDS;
    const int64_t n_tiles = (n + tile - 1) / tile;
    const size_t words = (size_t)passes * (RS_RADIX + 1 + (size_t)n_tiles * RS_RADIX) + 1;
    uint32_t* w = ar.alloc<uint32_t>(words);
    if (!w) return ar.err;
    uint32_t* ghist = w;                                   // [passes][256]
    uint32_t* counters = ghist + passes * RS_RADIX;        // [passes]
    uint32_t* err = counters + passes;                     // [1]
    uint32_t* status = err + 1;                            // [passes][n_tiles][256]
    cudaError_t e = cudaMemsetAsync(w, 0, words * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    int64_t hist_blocks = (n + OS_THREADS * 4 - 1) / (OS_THREADS * 4);  // ~4 keys per thread, at most 8 CTAs per SM
    if (hist_blocks > (int64_t)n_sm * 8) hist_blocks = (int64_t)n_sm * 8;
    uint32_t* perr = call_err ? call_err : err;
    launch_pdl(k_os_hist<K>, dim3((unsigned)(hist_blocks < 1 ? 1 : hist_blocks)), dim3(OS_THREADS), s, keys, n, passes, n_bits, ghist);
    count_launches(1);
    K* src_k = keys;
    uint32_t* src_v = vals;
    K* dst_k = keys_alt;
    uint32_t* dst_v = vals_alt;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        const int bits = n_bits - shift < 8 ? n_bits - shift : 8;
        launch_pdl(k_os_pass<K, ROUNDS>, dim3((unsigned)n_tiles), dim3(OS_THREADS), s, src_k, src_v, n, shift, (1u << bits) - 1u, ghist + p * RS_RADIX, status + (size_t)p * n_tiles * RS_RADIX, counters + p, perr, dst_k, dst_v, OS_SPIN_LIMIT);
        count_launches(1);
        K* tk = src_k;
        src_k = dst_k;
        dst_k = tk;
        uint32_t* tv = src_v;
        src_v = dst_v;
        dst_v = tv;
    }
    keys = src_k;
    vals = src_v;
    return cudaGetLastError();
}

// Keys per tile: 256 x ROUNDS, growing with n so that a pass has about one to two tiles per
// SM: fewer, larger tiles shorten the look-back chains, which dominate small passes (a 112k-key
// depth sort: 2 rounds 65 us, 4 rounds 56 us, 8 rounds 61 us for its 5 passes).
int onesweep_rounds(int64_t n, int n_sm) {
    const int64_t per_round = (int64_t)OS_THREADS * n_sm;
    return n <= per_round ? 1 : n <= 2 * per_round ? 2 : n <= 4 * per_round ? 4 : 8;
}

template <typename K>
cudaError_t onesweep(K*& keys, uint32_t*& vals, K* keys_alt, uint32_t* vals_alt, int64_t n, int n_bits,
                     uint32_t* call_err, Arena& ar, cudaStream_t s) {
    const int n_sm = sm_count();
    switch (onesweep_rounds(n, n_sm)) {
    case 1: return onesweep_impl<K, 1>(keys, vals, keys_alt, vals_alt, n, n_bits, call_err, n_sm, ar, s);
    case 2: return onesweep_impl<K, 2>(keys, vals, keys_alt, vals_alt, n, n_bits, call_err, n_sm, ar, s);
    case 4: return onesweep_impl<K, 4>(keys, vals, keys_alt, vals_alt, n, n_bits, call_err, n_sm, ar, s);
    default: return onesweep_impl<K, 8>(keys, vals, keys_alt, vals_alt, n, n_bits, call_err, n_sm, ar, s);
    }
}

// The passes of a sort whose digit counts the producer of the keys has already taken.  The input
// buffers are overwritten (they are one side of the ping-pong); the last pass writes (*keys_out,
// vals_out), and a null *keys_out takes whichever ping-pong buffer that pass does not read.
template <typename K, int ROUNDS>
cudaError_t counted_passes(K* keys, uint32_t* vals, K* keys_tmp, uint32_t* vals_tmp, K** keys_out,
                           uint32_t* vals_out, int64_t n, int n_bits, const uint32_t* hist, uint32_t* words,
                           uint32_t* call_err, cudaStream_t s) {
    const int passes = (n_bits + 7) / 8;
    const int64_t n_tiles = (n + (int64_t)OS_THREADS * ROUNDS - 1) / ((int64_t)OS_THREADS * ROUNDS);
    uint32_t* counters = words;         // [passes]
    uint32_t* status = words + passes;  // [passes][n_tiles][256]
    K* sk = keys;
    uint32_t* sv = vals;
    for (int p = 0; p < passes; ++p) {
        const bool last = p == passes - 1;
        K* dk = sk == keys ? keys_tmp : keys;
        uint32_t* dvv = sv == vals ? vals_tmp : vals;
        if (last) {
            if (*keys_out) dk = *keys_out;
            dvv = vals_out;
        }
        const int shift = 8 * p;
        const int bits = n_bits - shift < 8 ? n_bits - shift : 8;
        launch_pdl(k_os_pass<K, ROUNDS>, dim3((unsigned)n_tiles), dim3(OS_THREADS), s, (const K*)sk,
                   (const uint32_t*)sv, n, shift, (1u << bits) - 1u, hist + p * RS_RADIX,
                   status + (size_t)p * n_tiles * RS_RADIX, counters + p, call_err, dk, dvv, OS_SPIN_LIMIT);
        count_launches(1);
        sk = dk;
        sv = dvv;
    }
    *keys_out = sk;
    return cudaGetLastError();
}

template <typename K>
cudaError_t sort_counted(K* keys, uint32_t* vals, K* keys_tmp, uint32_t* vals_tmp, K*& keys_out, uint32_t* vals_out,
                         int64_t n, int n_bits, const uint32_t* hist, uint32_t* words, uint32_t* call_err, Arena& ar,
                         cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (n_bits <= 0 || n == 1) {
        if (!keys_out) keys_out = keys_tmp;
        cudaError_t e = cudaMemcpyAsync(keys_out, keys, sizeof(K) * (size_t)n, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vals_out, vals, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
        return e;
    }
    if (n >= (int64_t)OS_VAL || (n_bits + 7) / 8 > OS_MAX_PASSES) {
        // counts beyond the 30-bit status words: reduce-then-scan passes, then a copy to the outputs
        K* kk = keys;
        uint32_t* vv = vals;
        cudaError_t e = radix_impl<K>(kk, vv, keys_tmp, vals_tmp, n, n_bits, ar, s);
        if (e != cudaSuccess) return e;
        if (!keys_out) keys_out = kk;
        if (keys_out != kk) e = cudaMemcpyAsync(keys_out, kk, sizeof(K) * (size_t)n, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && vals_out != vv)
            e = cudaMemcpyAsync(vals_out, vv, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
        return e;
    }
    switch (onesweep_rounds(n, sm_count())) {
    case 1: return counted_passes<K, 1>(keys, vals, keys_tmp, vals_tmp, &keys_out, vals_out, n, n_bits, hist, words, call_err, s);
    case 2: return counted_passes<K, 2>(keys, vals, keys_tmp, vals_tmp, &keys_out, vals_out, n, n_bits, hist, words, call_err, s);
    case 4: return counted_passes<K, 4>(keys, vals, keys_tmp, vals_tmp, &keys_out, vals_out, n, n_bits, hist, words, call_err, s);
    default: return counted_passes<K, 8>(keys, vals, keys_tmp, vals_tmp, &keys_out, vals_out, n, n_bits, hist, words, call_err, s);
    }
}

}  // namespace

int64_t sort_counted_words(int64_t n, int n_bits) {
    const int passes = (n_bits + 7) / 8;
    const int64_t per_tile = (int64_t)OS_THREADS * onesweep_rounds(n, sm_count());
    const int64_t n_tiles = (n + per_tile - 1) / per_tile;
    return passes + (int64_t)passes * n_tiles * RS_RADIX;
}

cudaError_t sort_counted_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_tmp, uint32_t* vals_tmp,
                             uint64_t*& keys_out, uint32_t* vals_out, int64_t n, int n_bits, const uint32_t* hist,
                             uint32_t* words, uint32_t* call_err, Arena& ar, cudaStream_t s) {
    return sort_counted<uint64_t>(keys, vals, keys_tmp, vals_tmp, keys_out, vals_out, n, n_bits, hist, words,
                                  call_err, ar, s);
}

cudaError_t sort_counted_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp,
                             uint32_t*& keys_out, uint32_t* vals_out, int64_t n, int n_bits, const uint32_t* hist,
                             uint32_t* words, uint32_t* call_err, Arena& ar, cudaStream_t s) {
    return sort_counted<uint32_t>(keys, vals, keys_tmp, vals_tmp, keys_out, vals_out, n, n_bits, hist, words,
                                  call_err, ar, s);
}

uint32_t* spin_error_word() {
    void* p = nullptr;
    return cudaGetSymbolAddress(&p, g_spin_error) == cudaSuccess ? static_cast<uint32_t*>(p) : nullptr;
}

int sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 152;
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

// One tile of a one-sweep pass whose predecessor never publishes: the tile takes index 1 from a
// counter preset to 1, and tile 0's status words stay zero, so every look-back spin of the tile
// runs out of `spin_limit` reads.  The kernel then sets the call's flag and the device's
// wait-error word and finishes its (clamped) scatter, like a pass in production.  All buffers
// are sized for two tiles of one round; nothing waits without a bound.
cudaError_t debug_sort_timeout(int spin_limit, uint32_t* call_flag, uint32_t* device_flag, cudaStream_t s) {
    const int64_t n = 2 * OS_THREADS;
    uint32_t* w = nullptr;
    const size_t words = (size_t)n * 4 + RS_RADIX + 2 * RS_RADIX + 2;
    cudaError_t e = cudaMallocAsync(&w, words * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    uint32_t* keys = w;                        // [n]
    uint32_t* vals = keys + n;                 // [n]
    uint32_t* okeys = vals + n;                // [n]
    uint32_t* ovals = okeys + n;               // [n]
    uint32_t* goff = ovals + n;                // [256] zero: every digit starts at 0
    uint32_t* status = goff + RS_RADIX;        // [2][256] zero: tile 0 never publishes
    uint32_t* counter = status + 2 * RS_RADIX; // [1] = 1: the launched tile is tile 1
    uint32_t* err = counter + 1;               // [1]
    e = cudaMemsetAsync(w, 0, words * sizeof(uint32_t), s);
    const uint32_t one = 1u;
    if (e == cudaSuccess) e = cudaMemcpyAsync(counter, &one, sizeof(one), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_os_pass<uint32_t, 1><<<1, OS_THREADS, 0, s>>>(keys, vals, n, 0, 0xffu, goff, status, counter, err, okeys,
                                                         ovals, spin_limit);
        e = cudaGetLastError();
    }
    uint32_t h = 0, d = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(&d, g_spin_error, sizeof(d), 0, cudaMemcpyDeviceToHost, s);
    const uint32_t zero = 0u;
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_spin_error, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s);
    cudaFreeAsync(w, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *call_flag = h;
    *device_flag = d;
    return e;
}

cudaError_t scan_u32_to_u64(const uint32_t* in, uint64_t* out, int64_t n, uint64_t* total_dev, Arena& ar,
                            cudaStream_t s) {
    return scan_impl<uint32_t, uint64_t>(in, out, n, total_dev, ar, s);
}

cudaError_t scan_u32_to_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev, Arena& ar,
                            cudaStream_t s) {
    return scan_impl<uint32_t, uint32_t>(in, out, n, total_dev, ar, s);
}

// one-sweep passes while the counts fit the 30-bit status words, reduce-then-scan passes beyond
cudaError_t radix_sort_u64(uint64_t*& keys, uint32_t*& vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                           int n_bits, Arena& ar, cudaStream_t s, uint32_t* call_err) {
    if (n <= 1 || n_bits <= 0) return cudaSuccess;
    if (n < (int64_t)OS_VAL && (n_bits + 7) / 8 <= OS_MAX_PASSES)
        return onesweep<uint64_t>(keys, vals, keys_alt, vals_alt, n, n_bits, call_err, ar, s);
    return radix_impl<uint64_t>(keys, vals, keys_alt, vals_alt, n, n_bits, ar, s);
}

}  // namespace dv
