// Kernels of one BuildGram round (Sec. 3.3) over all active strings of a
// batch, and their host-side launchers.
//
// A round i reads the sequence T^i (bytes in round 1, uint32 ranks later) of
// the active strings, laid out back to back with offsets soff[0..k], and the
// fingerprints of its symbols (F^0 of the bytes in round 1; afterwards the
// fingerprint stream the previous round's rewrite wrote).  It runs:
//   k_tile_strings  per parse tile, the string holding its first position, and
//                   the bitmap of string starts
//   k_breaks   RandLMSPar break bits (Eq. rand_types) as a bitmap, 32
//              positions per thread
//   k_parse    per tile: the phrase starts (from the bitmap), a key per phrase
//              (its symbols when short, else a hash of its Eq. fast_hash
//              polynomial and its position) and its slot in the round's
//              phrase table, whose value is the smallest phrase index of the
//              content (content-confirmed, never by hash alone)
//   k_scan2    tile phrase counts -> global phrase indices (single pass)
//   k_strings  per-string phrase ranges; strings that became one phrase retire
//   k_mark, k_popscan, k_rank
//              first-occurrence naming: the first occurrences of the new
//              phrases are marked in a bitmap over phrase indices, and a
//              phrase's rank is the number of marks before its own
//   k_scan2    rule lengths -> right-hand-side offsets
//   k_rules    the level-i rules in rank order: rhs, rhs_off and F^i, and the
//              (F^i, rank) pair of every table slot
//   k_rewrite  T^{i+1}[p] = rank of phrase p and its fingerprint, compacting
//              retired strings
// A short round (at most kSmallTiles tiles) runs the same steps as two
// cooperative launches instead: k_parse_small (tile strings to strings) and
// k_naming_small (marks to rewrite), with grid barriers between the steps.
// Every kernel of the round starts with pdl_wait(): it is launched with
// programmatic dependent launch after the one before it.
#include <algorithm>
#include <utility>

#include "lcg_dev.cuh"
#include "lcg_internal.h"
#include "table.cuh"

namespace lcg {

constexpr u32 kResidentBit = 0x80000000u;  // P_slot entry names a resident rank

template <typename T>
struct FpSource;  // fingerprint of a symbol

template <>
struct FpSource<unsigned char> {
    const u32* F;  // shared-memory copy of F^0
    __device__ __forceinline__ u32 operator()(unsigned char s) const { return F[s]; }
};
template <>
struct FpSource<u32> {
    const u32* F;  // F^{i-1} in global memory
    __device__ __forceinline__ u32 operator()(u32 s) const { return __ldg(F + s); }
};

// Sizes of a round: from the device when the round was enqueued without a
// host synchronisation, else from the arguments.
__device__ __forceinline__ u64 round_n(const RoundArgs& a) { return a.d_n ? *a.d_n : a.n; }
__device__ __forceinline__ u32 round_k(const RoundArgs& a) { return a.d_k ? (u32)*a.d_k : a.k; }

// A round stops as soon as it, or the round before it, has failed (an error,
// or a phrase table past its load limit): its inputs and buffers can no longer
// be trusted, and the host discards or reruns it.  Called by every thread of a
// block; the answer is the same for the whole block.
__device__ bool round_halted(const RoundArgs& a) {
    __shared__ int s_halt;
    __syncthreads();
    if (threadIdx.x == 0) {
        bool h = vload(&a.ds->error) != 0 || vload(&a.ds->overflow) != 0;
        if (a.ds_prev) h = h || vload(&a.ds_prev->error) != 0 || vload(&a.ds_prev->overflow) != 0;
        s_halt = h ? 1 : 0;
    }
    __syncthreads();
    return s_halt != 0;
}

// index of the string holding position `pos`: largest j with soff[j] <= pos
__device__ __forceinline__ u32 string_of(const u64* soff, u32 k, u64 pos) {
    u32 lo = 0, hi = k;  // answer in [lo, hi)
    while (hi - lo > 1) {
        const u32 mid = (lo + hi) >> 1;
        if (__ldg(soff + mid) <= pos) lo = mid; else hi = mid;
    }
    return lo;
}

// --------------------------------------------------------------------------
// k_parse
// --------------------------------------------------------------------------
//
// Persistent blocks take tiles of TP positions.  A tile's symbols (and kHalo
// more) and its words of the break bitmap are staged in shared memory (byte
// rounds read the next tile's into registers while parsing the current one);
// the phrase starts are listed in order by a block scan.  Each phrase gets a
// key: its symbols packed exactly when they fit in 124 bits, else a hash of
// its polynomial fingerprint H (Eq. fast_hash) with its length and position,
// confirmed by comparing contents.  It is looked up first in the resident
// level (when parsing against a resident grammar), then in the round's table,
// where a new content is claimed.  In byte rounds a per-block cache of packed
// phrases (kept across the block's tiles) answers most lookups; the phrases
// that miss are queued and looked up together, with full warps.  The slot of
// phrase q of tile t goes to P_slot[pslot_base(t) + q] (its order key is
// t * TP + q); new entries
// (claims) are listed in shared memory and appended to the round's claim list
// every few tiles.

constexpr int kParseThreads = 256;
// Positions per parse tile, TP: 1024, 2048 or 4096 (the default), a launch
// parameter (lcg_tuning.parse_tile) that every kernel of a round reads from
// RoundArgs::tp; k_parse is compiled for each.
constexpr int kTPMin = 1024, kTPMax = 4096;
// Rounds of at most kSmallTiles tiles of kTPMin positions run as two
// cooperative launches (parse; naming and rewrite) whose steps are separated
// by grid barriers, instead of eleven launches: launch latency, not work,
// bounds such rounds.
constexpr u64 kSmallTiles = 128;
constexpr int kHalo = 64;          // positions staged past the tile end

// Where the phrase slots of parse tile t begin in P_slot.  Every phrase but a
// string's first is at least two symbols long, so a tile of TP positions in
// which s strings start holds at most TP / 2 + 1 + s phrases.  With j0(t)
// the string holding the tile's first position (tile_str[t]), s is at most
// j0(t + 1) - j0(t) + 1, so tile t's slots can begin at t (TP / 2 + 2) + j0(t).
__device__ __forceinline__ u64 pslot_base(u64 t, u32 j0, u32 tp) { return t * (u64)(tp / 2 + 2) + j0; }

// Tile order of the rank rounds' parse and rewrite: with `stripes` = k > 1
// the round's tiles are cut into k equal stripes and taken interleaved
// (stripe 0's first tile, stripe 1's first tile, ..., then every stripe's
// second tile), so that strings which are near-copies of one another at the
// same offsets (k assemblies of one genome) are parsed side by side and the
// later copies find the first copy's new table entries still in L2.  Logical
// tile l in [0, k * ceil(T / k)) names tile (l % k) * ceil(T / k) + l / k, or
// nothing (>= T).  Phrase order keys stay tile * TP + q, so the result does
// not depend on the order.
__device__ __forceinline__ u64 stripe_tiles(u64 ntiles, u32 stripes) {
    if (stripes <= 1) return ntiles;
    const u64 per = (ntiles + stripes - 1) / stripes;
    return per * stripes;
}
__device__ __forceinline__ u64 stripe_tile(u64 l, u64 ntiles, u32 stripes) {
    if (stripes <= 1) return l;
    const u64 per = (ntiles + stripes - 1) / stripes;
    return (l % stripes) * per + l / stripes;
}
constexpr int kCacheBits = 11;
constexpr int kCacheSlots = 1 << kCacheBits;  // per-block phrase cache (byte rounds)
constexpr int kCacheProbes = 8;
// New table entries of a block are listed in shared memory and appended to
// the round's claim list once the buffer is half full, or in rank rounds once
// another tile could overflow it (a tile claims at most TP entries), and
// after the block's last tile, so that the global counter is touched every
// few tiles only.
constexpr int kClaimBufB = 512;   // byte rounds (shared memory also holds the phrase cache)
constexpr int kClaimBufR = 4096;  // rank rounds
// Byte rounds: phrases that miss the block's cache are queued with their keys
// and looked up in the global table together once the queue is half full, so
// that full warps run the long lookup path, every few tiles.
constexpr int kMissBuf = 256;
constexpr int kMissFlushDefault = 64;  // queued misses that trigger a lookup pass
constexpr u64 kOkeyBits = 44;  // order keys are below 2^44
// Table slots read per round trip.  One: a random DRAM read costs per 32-byte
// sector (one slot), and at the default table load of 0.35 most lookups end
// at their home slot; reading the home slot's group of two took more DRAM
// sectors per lookup and was slower in the rank rounds, where those random
// sectors bound k_parse.
constexpr int kProbeGroup = 1;
// Long phrases (hashed keys) in rank rounds: fingerprints read per round
// trip for H, and symbols per round trip when a match is confirmed by content
// (byte rounds read staged fingerprints and take one at a time).
constexpr int kHornerBatchR = 8;
constexpr int kCompareBatchR = 4;
// Phrases longer than kLongLen (N-runs of DNA, repeated text) are hashed and
// compared by a whole warp after the tile's other phrases: a thread alone
// would spend a round trip per symbol on them while its block waits.  Their
// starts are more than kLongLen apart, so a tile holds at most
// TP / (kLongLen + 1) + 1.
constexpr int kLongLen = 32;

// Load n_sym symbols of type V from src (16-byte aligned when `vec`) into the
// shared array dst, with every 16-byte load issued before any is stored.
template <int SP, typename V>
__device__ __forceinline__ void stage_vec(V* dst, const V* src, int n_sym, bool vec) {
    constexpr int PER = 16 / sizeof(V);
    constexpr int NV = (SP + PER - 1) / PER;
    constexpr int IT = (NV + kParseThreads - 1) / kParseThreads;
    uint4 buf[IT];
#pragma unroll
    for (int it = 0; it < IT; it++) {
        const int x0 = (threadIdx.x + it * kParseThreads) * PER;
        if (x0 + PER <= n_sym && vec) {
            buf[it] = __ldcs(reinterpret_cast<const uint4*>(src + x0));  // streamed once: evict first
        } else if (x0 < n_sym) {
            V tmp[PER];
#pragma unroll
            for (int e = 0; e < PER; e++) tmp[e] = (x0 + e < n_sym) ? src[x0 + e] : (V)0;
            buf[it] = *reinterpret_cast<const uint4*>(tmp);
        }
    }
#pragma unroll
    for (int it = 0; it < IT; it++) {
        const int x0 = (threadIdx.x + it * kParseThreads) * PER;
        if (x0 < n_sym) *reinterpret_cast<uint4*>(dst + x0) = buf[it];
    }
}

// --------------------------------------------------------------------------
// k_breaks: the round's break bitmap (Eq. rand_types)
// --------------------------------------------------------------------------
//
// A phrase starts at x when x starts a string, or f[x-1] > f[x] and x has
// type S: the first fingerprint right of x (within the string) that differs
// from f[x] is larger than f[x].  Thread t of a block step owns the 32
// positions of bitmap word t and works on bit masks: gt / lt mark positions
// whose right neighbour (in the string) is larger / smaller, stop marks
// positions whose right neighbour starts a string (or is past the end).  A
// position's type is decided by the first of these at or above it, so the S
// mask is gt spread down over the undecided positions (five doubling steps).
// Positions above the thread's last decision take the type of the next
// thread's first position, found through per-thread summaries; past the block
// step, the type of the next step's first position.  Then breaks = starts |
// ((lt << 1) & S), bit 0 using f of the position before.
//
// A run of equal fingerprints can span many block steps (N-runs of DNA).
// Block steps are therefore taken in decreasing order from a counter, and
// each publishes the type of its first position (its "head") as soon as its
// masks are known: decided, or "open" when the whole step is one run.  A step
// whose last position is undecided reads the heads of the steps after it,
// skipping open ones, until one is decided (a look-ahead over steps that were
// all taken before it, so every wait ends); an open step then publishes the
// type it found as its head.  Each step reads its own positions once, however
// long the run.

constexpr int kBrkThreads = 256;
constexpr u64 kBrkSpan = (u64)kBrkThreads * 32;  // positions per block step
static_assert(kBrkSpan % kTPMax == 0, "a block step starts a parse tile");

// Head of block step b in the look-ahead words: (epoch << 8) | (state << 2) |
// type, state 1 = open, 2 = decided.
__device__ __forceinline__ void brk_publish(u64* heads, u64 b, u64 epoch, u32 state, u32 type) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(heads + b), "l"((epoch << 8) | (state << 2) | type)
                 : "memory");
}

// Type of the first position of step j (the run continues into it), looking
// further right past open steps.  `none` is the type past the last step.
__device__ u32 brk_lookahead(const u64* heads, u64 j, u64 nsteps, u64 epoch, u32 none, DevStatus* ds) {
    for (; j < nsteps; j++) {
        u64 it = 0;
        u32 backoff = 32;
        while (true) {
            u64 w;
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(heads + j) : "memory");
            if ((w >> 8) == epoch) {
                if (((w >> 2) & 3u) == 2u) return (u32)(w & 3u);
                break;  // open: one run throughout, look at the next step
            }
            if (++it > kSpinLimit || vload(&ds->error) != 0) {
                set_error(ds, kErrTimeout);
                return none;
            }
            __nanosleep(backoff);
            if (backoff < 256) backoff <<= 1;
        }
    }
    return none;
}

// Spread the bits of `src` down over the positions of `pass` (positions that
// take the value of the position above): bit i of the result is src[j] for
// the first j >= i with pass[j] == 0, when that j is at most 31.
__device__ __forceinline__ u32 spread_down(u32 src, u32 pass) {
    u32 y = src, m = pass;
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
        y |= (y >> k) & m;
        m &= m >> k;
    }
    return y;
}

// Kernel bodies are device functions: k_X launches body_X on a grid, and the
// short rounds' cooperative kernels (k_parse_small, k_naming_small) run several of
// them in one launch.
template <typename T>
__device__ __forceinline__ void body_breaks(const RoundArgs& a, u64 nblocks) {
    pdl_wait();
    constexpr bool kByte = sizeof(T) == 1;
    constexpr u32 kTypeU = 0, kTypeS = 1, kTypeL = 2, kUndecided = 3;
    constexpr int SW = kBrkThreads;  // string-start words of a step
    __shared__ u32 sF0[kByte ? 256 : 1];
    __shared__ u32 sst[SW + 1];      // string starts at base .. base + kBrkSpan
    __shared__ u32 sfirst[kBrkThreads];  // type of each thread's first position
    __shared__ u64 s_step;
    __shared__ u32 s_open, s_carry;
    if (round_halted(a)) return;
    const T* S = (const T*)a.S;
    const u32* Sf = a.Sf;
    const u64 n = round_n(a);
    const int tid = threadIdx.x, lane = tid & 31;
    if constexpr (kByte)
        for (int x = tid; x < 256; x += kBrkThreads) sF0[x] = a.Fprev[x];
    auto fpos = [&](u64 x) -> u32 {  // fingerprint of position x < n
        if constexpr (kByte) return sF0[S[x]]; else return __ldg(Sf + x);
    };
    const bool aligned = kByte ? (reinterpret_cast<unsigned long long>(S) & 15) == 0
                               : (reinterpret_cast<unsigned long long>(Sf) & 15) == 0;
    nblocks = min(nblocks, (n + kBrkSpan - 1) / kBrkSpan);
    if (blockIdx.x >= nblocks && blockIdx.x > 0) return;  // more blocks than steps: no counter traffic
    u64* heads = a.heads;
    const int warp = tid >> 5;
    while (true) {
        // the next block step, in decreasing order (the counter starts at 0 every round)
        if (tid == 0) {
            const u64 t = atomicAdd(&a.ds->aux[0], 1ull);
            s_step = t < nblocks ? nblocks - 1 - t : ~0ull;
        }
        __syncthreads();  // also: sF0 loaded
        const u64 b = s_step;
        if (b == ~0ull) break;
        const u64 base = b * kBrkSpan;
        const u64 bend = min(base + kBrkSpan, n);
        // string starts (bitmap of k_tile_strings; n counts as one)
        for (int w = tid; w <= SW; w += kBrkThreads) {
            const u64 gw = base / 32 + (u64)w;
            sst[w] = gw < a.sbm_words ? __ldg(a.sbm + gw) : 0u;
        }
        const u64 x0 = base + 32ull * (u64)tid;
        u32 f[32];
        if (aligned && x0 + 32 <= n) {
            if constexpr (kByte) {
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const uint4 v = __ldcs(reinterpret_cast<const uint4*>(S + x0 + 16 * h));
                    const u32 w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int i = 0; i < 16; i++) f[16 * h + i] = sF0[(w[i >> 2] >> (8 * (i & 3))) & 0xFFu];
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const uint4 v = __ldcs(reinterpret_cast<const uint4*>(Sf + x0 + 4 * q));
                    f[4 * q] = v.x;
                    f[4 * q + 1] = v.y;
                    f[4 * q + 2] = v.z;
                    f[4 * q + 3] = v.w;
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < 32; i++) f[i] = (x0 + i < n) ? fpos(x0 + i) : 0u;
        }
        // f of the position after the thread's last, and of the one before its first
        u32 fnext = __shfl_down_sync(0xffffffffu, f[0], 1);
        u32 fprev = __shfl_up_sync(0xffffffffu, f[31], 1);
        if (lane == 31 && x0 + 32 < n) fnext = fpos(x0 + 32);
        if (lane == 0 && x0 > 0 && x0 - 1 < n) fprev = fpos(x0 - 1);
        __syncthreads();  // sst loaded
        const u32 st = sst[tid];                      // starts at x0 .. x0 + 31
        const u32 st_next = (sst[tid + 1] & 1u);      // start at x0 + 32
        // masks over the thread's positions: right neighbour larger, smaller,
        // or a string start / the end of the sequence
        const u32 stop = (st >> 1) | (st_next << 31);
        u32 gt = 0, lt = 0;
#pragma unroll
        for (int i = 0; i < 31; i++) {
            gt |= (u32)(f[i + 1] > f[i]) << i;
            lt |= (u32)(f[i + 1] < f[i]) << i;
        }
        gt |= (u32)(fnext > f[31]) << 31;
        lt |= (u32)(fnext < f[31]) << 31;
        gt &= ~stop;
        lt &= ~stop;
        const u32 dec = gt | lt | stop;  // positions whose type is decided here
        u32 sm = spread_down(gt, ~dec);
        u32 lm = spread_down(lt, ~dec);
        // type of the thread's first position (or undecided: one run throughout)
        sfirst[tid] = dec == 0 ? kUndecided : (sm & 1u) ? kTypeS : (lm & 1u) ? kTypeL : kTypeU;
        const bool open = dec != (u32)~0u && ((dec >> 31) & 1u) == 0;  // positions above the last decision
        if (tid == kBrkThreads - 1) s_open = open ? 1u : 0u;
        __syncthreads();
        if (warp == 0) {
            // the step's head: the type of the first thread whose first position is decided
            u32 head = kUndecided;
            for (int c = 0; c < kBrkThreads / 32; c++) {
                const u32 v = sfirst[c * 32 + lane];
                const unsigned m = __ballot_sync(0xffffffffu, v != kUndecided);
                if (m) {
                    head = __shfl_sync(0xffffffffu, v, __ffs(m) - 1);
                    break;
                }
            }
            if (lane == 0) {
                brk_publish(heads, b, a.brk_epoch, head == kUndecided ? 1u : 2u, head == kUndecided ? 0u : head);
                // type of the next step's first position (the last thread's run goes on there)
                u32 carry = kTypeU;
                if (bend < n && s_open) carry = brk_lookahead(heads, b + 1, nblocks, a.brk_epoch, kTypeU, a.ds);
                if (head == kUndecided) brk_publish(heads, b, a.brk_epoch, 2u, carry);
                s_carry = carry;
            }
        }
        __syncthreads();
        if (open) {
            // positions above the last decision take the type of position x0 + 32:
            // the first decided thread after this one, else the next step's head
            u32 carry = s_carry;
            for (int t = tid + 1; t < kBrkThreads; t++) {
                const u32 c = sfirst[t];
                if (c != kUndecided) {
                    carry = c;
                    break;
                }
            }
            const int hi = 31 - __clz(dec | 1u);  // highest decided position (or 0)
            const u32 top = dec == 0 ? ~0u : ~((2u << hi) - 1u);
            if (carry == kTypeS) sm |= top;
            if (carry == kTypeL) lm |= top;
        }
        u32 bits = st | ((lt << 1) & sm);
        if (fprev > f[0] && (sm & 1u)) bits |= 1u;
        if (x0 < bend) {
            if (bend - x0 < 32) bits &= (1u << (bend - x0)) - 1u;
            a.brk[x0 >> 5] = bits;
        }
        __syncthreads();
    }
}

// Exclusive scan of one 32-bit value per thread of a kParseThreads block, with
// one barrier: every warp scans the warp totals itself.  `s_wsum` (one word
// per warp) must not be written again before all threads have returned.
__device__ __forceinline__ u32 block_scan32(u32 x, u32& total, u32* s_wsum) {
    constexpr int NW = kParseThreads / 32;
    const u32 lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    u32 incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
    }
    if (lane == 31) s_wsum[wid] = incl;
    __syncthreads();
    const u32 w = lane < (u32)NW ? s_wsum[lane] : 0u;
    u32 wi = w;
#pragma unroll
    for (int o = 1; o < NW; o <<= 1) {
        const u32 y = __shfl_up_sync(0xffffffffu, wi, o);
        if ((int)lane >= o) wi += y;
    }
    total = __shfl_sync(0xffffffffu, wi, NW - 1);
    return __shfl_sync(0xffffffffu, wi - w, wid) + incl - x;
}

template <typename T, int TP>
__device__ __forceinline__ void body_parse(const RoundArgs& a, u64 ntiles) {
    pdl_wait();
    constexpr int kSP = TP + kHalo;  // staged positions
    constexpr int NWS = kSP / 32;    // staged break words
    constexpr int NWT = TP / 32;     // tile break words
    constexpr int kLongBuf = TP / (kLongLen + 1) + 1;
    constexpr bool kByte = sizeof(T) == 1;
    constexpr bool kLocal = kByte;
    static_assert(NWT <= kParseThreads, "one tile word per thread");
    constexpr int kClaimBuf = kByte ? kClaimBufB : kClaimBufR;
    constexpr int kHornerBatch = kByte ? 1 : kHornerBatchR;
    constexpr int kCompareBatch = kByte ? 1 : kCompareBatchR;

    __shared__ u32 sF0[kByte ? 256 : 1];
    // bytes of tile positions (and 32 more: packed keys read whole 8-byte words past a phrase)
    __shared__ __align__(16) unsigned char sb[kByte ? kSP + 32 : 16];
    __shared__ __align__(16) u32 sT[kByte ? 4 : kSP];             // ranks of tile positions
    __shared__ u32 sbits[NWS];
    __shared__ u32 swp[NWT];
    __shared__ unsigned short sP[TP];
    // byte rounds: per-block cache of phrase (packed bytes) -> slot, kept across
    // the block's tiles (its entries always come from earlier tiles)
    __shared__ u64 ckey[kLocal ? kCacheSlots : 1];
    __shared__ u32 cval[kLocal ? kCacheSlots : 1];
    __shared__ u32 sClaim[kClaimBuf];
    __shared__ u32 s_wsum[kParseThreads / 32];
    // byte rounds: queued cache misses: key, and order key | (cache slot + 1) << kOkeyBits
    // (half as many with 4096-position tiles, whose staged bytes and phrase
    // list take that room: the block's static shared memory stays under 48 KB)
    constexpr int kMissCap = TP >= 4096 ? kMissBuf / 2 : kMissBuf;
    __shared__ Key128 sMissKey[kLocal ? kMissCap : 1];
    __shared__ u64 sMissOk[kLocal ? kMissCap : 1];
    __shared__ u64 sMissPs[kLocal ? kMissCap : 1];  // where the queued phrase's slot goes in P_slot
    __shared__ u32 s_nmiss;
    __shared__ unsigned short sLong[kLongBuf];  // tile offsets (q) of the tile's long phrases
    __shared__ u32 s_nlong;
    __shared__ u64 s_tail_end;
    __shared__ u32 s_nclaim;
    __shared__ u64 s_claim_len;
    __shared__ u64 s_claim_base;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T* S = (const T*)a.S;
    const u64 n = round_n(a);
    const u32 kact = round_k(a);
    const u64 nwords = (n + 31) / 32;  // words of the break bitmap
    ntiles = min(ntiles, (n + TP - 1) / TP);
    FpSource<T> fp;
    if constexpr (kByte) {
        for (int x = tid; x < 256; x += kParseThreads) sF0[x] = a.Fprev[x];
        fp.F = sF0;
    } else {
        fp.F = a.Fprev;
    }
    const ContentTable bt{(Slot*)a.tab, a.tab_cap};
    const ContentTable rt{(Slot*)a.rtab, a.rtab_cap};
    if constexpr (kLocal) {
        for (int x = tid; x < kCacheSlots; x += kParseThreads) {
            ckey[x] = kEmpty;
            cval[x] = ~0u;
        }
    }
    if (tid == 0) {
        s_nclaim = 0;
        s_claim_len = 0;
        s_nmiss = 0;
        s_nlong = 0;
    }

    // persistent blocks: tiles blockIdx.x, blockIdx.x + gridDim.x, ...  Tiles
    // do not depend on one another.
    // Byte rounds: a tile's bytes (16 per thread and load), break words and
    // string index are read into registers while the block parses the tile
    // before it.
    constexpr int kFetch = (kSP + 16 * kParseThreads - 1) / (16 * kParseThreads);  // 16-byte loads per thread
    static_assert(NWS <= kParseThreads, "one break word per thread");
    uint4 pf_sym[kFetch];
#pragma unroll
    for (int f = 0; f < kFetch; f++) pf_sym[f] = make_uint4(0u, 0u, 0u, 0u);
    u32 pf_bits = 0, pf_j0 = 0;
    auto fetch = [&](u64 tl) {
        const u64 f0 = tl * (u64)TP;
        const int fns = (int)(min(f0 + (u64)kSP, n) - f0);
        const unsigned char* src = (const unsigned char*)S + f0;
#pragma unroll
        for (int f = 0; f < kFetch; f++) {
            const int x0 = (tid + f * kParseThreads) * 16;
            if (x0 + 16 <= fns && (reinterpret_cast<unsigned long long>(src) & 15) == 0) {
                pf_sym[f] = __ldcs(reinterpret_cast<const uint4*>(src + x0));  // streamed once: evict first
            } else if (x0 < fns) {
                unsigned char tmp[16];
#pragma unroll
                for (int e = 0; e < 16; e++) tmp[e] = (x0 + e < fns) ? src[x0 + e] : (unsigned char)0;
                pf_sym[f] = *reinterpret_cast<const uint4*>(tmp);
            }
        }
        const u64 gw = f0 / 32 + (u64)tid;
        pf_bits = (tid < NWS && gw < nwords) ? __ldg(a.brk + gw) : 0u;
        pf_j0 = a.tile_str[tl];
    };

    u64 iter = 0;
    // rank rounds may take their tiles in stripes (stripe_tile); byte rounds in order
    const u32 stripes = kByte ? 1u : a.stripes;
    const u64 nlog = stripe_tiles(ntiles, stripes);
    for (u64 lt = blockIdx.x; lt < nlog; lt += gridDim.x, iter++) {
        if ((iter & 15) == 0 && round_halted(a)) break;
        const u64 tile = stripe_tile(lt, ntiles, stripes);
        const bool last = lt + gridDim.x >= nlog;  // the block's last tile
        if (tile >= ntiles) continue;  // no tile here (claims still buffered are flushed after the loop)
        const u64 t0 = tile * (u64)TP;
        const u64 t_end = min(t0 + (u64)TP, n), s_end = min(t0 + (u64)kSP, n);
        const int ns = (int)(s_end - t0), nt = (int)(t_end - t0);

        // 1. stage the tile's symbols (bytes in round 1, ranks afterwards) and
        //    its break words (k_breaks)
        u32 j0;  // string holding t0
        if constexpr (kByte) {
            if (iter == 0) fetch(tile);
#pragma unroll
            for (int f = 0; f < kFetch; f++) {
                const int x0 = (tid + f * kParseThreads) * 16;
                if (x0 < ns) *reinterpret_cast<uint4*>(sb + x0) = pf_sym[f];
            }
            if (tid < NWS) sbits[tid] = pf_bits;
            j0 = pf_j0;
            if (tile + gridDim.x < ntiles) fetch(tile + gridDim.x);  // byte rounds: in order
        } else {
            j0 = a.tile_str[tile];
            stage_vec<kSP, u32>(sT, S + t0, ns, (reinterpret_cast<unsigned long long>(S + t0) & 15) == 0);
            for (int w = tid; w < NWS; w += kParseThreads) {
                const u64 gw = t0 / 32 + (u64)w;
                sbits[w] = gw < nwords ? __ldg(a.brk + gw) : 0u;
            }
        }
        // offsets of the strings from j0 on, for step 5 (read now, used at the tile's end)
        const u64 s_first = (warp == 0 && j0 + lane < kact) ? __ldg(a.soff + j0 + lane) : ~0ull;
        const u64 pb0 = pslot_base(tile, j0, TP);  // the tile's phrase slots in P_slot
        __syncthreads();

        // 3. phrase starts of the tile, in order: kTPW threads per break
        //    word, kBPT bits each
        constexpr int kTPW = kParseThreads / NWT, kBPT = 32 / kTPW;
        static_assert(kTPW * NWT == kParseThreads && kTPW * kBPT == 32 && kBPT < 32, "threads per tile word");
        const int wq = tid / kTPW, bq = (tid % kTPW) * kBPT;
        u32 word = sbits[wq];
        if (wq * 32 >= nt) word = 0;
        else if (nt - wq * 32 < 32) word &= (1u << (nt - wq * 32)) - 1u;
        const u32 part = (word >> bq) & ((1u << kBPT) - 1u);
        u32 cnt;
        const u32 poff = block_scan32((u32)__popc(part), cnt, s_wsum);
        if (tid % kTPW == 0) swp[wq] = (u32)poff;
        {
            u32 m = part, o = (u32)poff;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                sP[o++] = (unsigned short)(wq * 32 + bq + b);
            }
        }
        if (tid == 0) {
            // end of the tile's last phrase: the first phrase start at or after t_end
            u64 e = n;
            bool found = false;
            for (int w = nt >> 5; w < (ns + 31) >> 5 && !found; w++) {
                u32 m = sbits[w];
                if (w == (nt >> 5)) m &= ~((1u << (nt & 31)) - 1u);
                if (m) { e = t0 + (u64)(w * 32 + __ffs(m) - 1); found = true; }
            }
            // past the staged words (s_end < n is then a multiple of 32): the
            // bitmap in global memory
            for (u64 gw = s_end / 32; !found && s_end < n && gw < nwords; gw++) {
                const u32 m = __ldg(a.brk + gw);
                if (m) { e = min(n, gw * 32 + (u64)(__ffs(m) - 1)); found = true; }
            }
            s_tail_end = e;
        }
        __syncthreads();

        // 4. lookups.  A phrase's order key is tile * TP + q: it orders phrases
        //    like their global index.
        const u64 tail = s_tail_end - t0;
        const u32 cntq = (u32)cnt;
        const u64 okey0 = tile * (u64)TP;
        auto phrase_end = [&](u32 q) -> u64 { return (q + 1 < cntq) ? (u64)sP[q + 1] : tail; };
        auto sym = [&](u64 x) -> u32 {  // symbol at tile offset x
            if (x < (u64)ns) {
                if constexpr (kByte) return (u32)sb[x]; else return sT[x];
            }
            return (u32)S[t0 + x];
        };
        // the slot of phrase q = [st, en); *claimed when this call made the entry
        // key of phrase [st, en) (tile offsets); *ok = false for one too long
        auto make_key = [&](u64 st, u64 en, bool* ok) -> Key128 {
            const u64 len = en - st;
            *ok = len <= kMaxPhraseLen;
            if (!*ok) {
                set_error(a.ds, kErrPhraseLong);
                return Key128{0, 0};
            }
            if (len > inline_max(a.sym_w)) {
                // H = sum_j F[Q_j] c^{j-1} mod p, by Horner from the last symbol;
                // the fingerprints (staged F^0 of bytes, or the round's
                // fingerprint stream) are read kHornerBatch at a time
                u64 H = 0;
                for (u64 x = en; x > st;) {
                    const u64 c = min((u64)kHornerBatch, x - st);
                    u32 f[kHornerBatch];
#pragma unroll
                    for (int u = 0; u < kHornerBatch; u++) {
                        if ((u64)u < c) {
                            if constexpr (kByte) f[u] = fp((unsigned char)sym(x - 1 - u));
                            else f[u] = __ldg(a.Sf + t0 + x - 1 - u);
                        } else {
                            f[u] = 0;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kHornerBatch; u++)
                        if ((u64)u < c) H = addmod61(mulmod61(H, a.lh.c), (u64)f[u]);
                    x -= c;
                }
                return key_hashed(H, len, t0 + st);
            }
            return key_inline([&](u64 j) { return sym(st + j); }, len, a.sym_w);
        };
        // The slot of a phrase given its key and order key (a hashed key names
        // the phrase's position in S); *claimed when this call made the entry.
        auto lookup_key = [&](const Key128& key, u64 okey, bool* claimed) -> u32 {
            *claimed = false;
            const bool hashed = key_is_hashed(key);
            const u64 len = key_len(key), pos = key.lo;
            if (rt.cap) {
                const u64 r = table_find(rt, key, hashed, [&](u64 rank) {
                    const u64 o = a.rrhs_off[rank];
                    for (u64 j = 0; j < len; j++)
                        if ((u32)S[pos + j] != a.rrhs[o + j]) return false;
                    return true;
                });
                if (r != ~0ull) return kResidentBit | (u32)r;
            }
            return (u32)table_claim_or_find<kByte ? 1 : kProbeGroup>(bt, key, hashed, okey, [&](u64 ref) {
                // both contents in global memory, kCompareBatch symbols per round trip
                for (u64 j = 0; j < len; j += kCompareBatch) {
                    T x[kCompareBatch], y[kCompareBatch];
#pragma unroll
                    for (int u = 0; u < kCompareBatch; u++) {
                        const bool in = j + u < len;
                        x[u] = in ? S[ref + j + u] : (T)0;
                        y[u] = in ? S[pos + j + u] : (T)0;
                    }
#pragma unroll
                    for (int u = 0; u < kCompareBatch; u++)
                        if (x[u] != y[u]) return false;
                }
                return true;
            }, claimed, a.ds);
        };
        auto lookup = [&](u32 q, u64 st, u64 en, bool* claimed) -> u32 {
            bool ok;
            const Key128 key = make_key(st, en, &ok);
            if (!ok) {
                *claimed = false;
                return ~0u;
            }
            return lookup_key(key, okey0 + q, claimed);
        };
        // New entries join the block's claim buffer (or, when it is full, the
        // round's list at once).  claim_warp is called by all lanes of a warp
        // together and makes one shared-memory update per warp.
        auto claim_one = [&](u32 slot, u64 len, u32 c) {
            if (c < (u32)kClaimBuf) {
                sClaim[c] = slot;
            } else {
                const u64 g = atomicAdd(&a.ds->claims, 1ull);
                if (g < bt.cap) a.claims[g] = slot;
            }
        };
        auto claim_warp = [&](bool claimed, u32 slot, u64 len) {
            const unsigned m = __ballot_sync(0xffffffffu, claimed);
            if (m == 0) return;
            u64 sum = claimed ? len : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            const int leader = __ffs(m) - 1;
            u32 base = 0;
            if (lane == leader) {
                base = atomicAdd(&s_nclaim, (u32)__popc(m));
                atomicAdd(&s_claim_len, sum);
            }
            base = __shfl_sync(0xffffffffu, base, leader);
            if (claimed) claim_one(slot, len, base + (u32)__popc(m & ((1u << lane) - 1u)));
        };
        auto claim_single = [&](u32 slot, u64 len) {
            atomicAdd(&s_claim_len, len);
            claim_one(slot, len, atomicAdd(&s_nclaim, 1u));
        };
        auto defer_long = [&](u32 q) {
            const u32 x = atomicAdd(&s_nlong, 1u);
            if (x < (u32)kLongBuf) sLong[x] = (unsigned short)q;
            else set_error(a.ds, kErrCapacity);  // not reached: long phrases start > kLongLen apart
        };

        if constexpr (kLocal) {
            // Short phrases go through the block's cache.  Its entries come
            // from earlier tiles of the block, whose phrases precede this
            // tile's: a hit needs nothing more.  Misses are queued with their
            // keys and looked up in the global table together once the queue
            // is half full (and after the block's last tile).
            const u64* sb64 = reinterpret_cast<const u64*>(sb);
            // packed bytes of a phrase of length <= 7 inside the staged bytes
            auto short_key = [&](u32 st, u32 len) -> u64 {
                const u32 w = st >> 3, sh = (st & 7) * 8;
                const u64 lo = sb64[w], hi = sb64[w + 1];
                const u64 v = sh ? (lo >> sh) | (hi << (64 - sh)) : lo;
                return ((u64)len << 56) | (v & ((1ull << (8 * len)) - 1));
            };
            // the inline key of a phrase of length <= kInlineMax inside the staged
            // bytes: its bytes as one little-endian number B, B mod 2^60 (with
            // the length above) in hi and B >> 60 in lo (the layout of
            // key_inline for 8-bit symbols)
            auto byte_key = [&](u32 st, u32 len) -> Key128 {
                const u32 w = st >> 3, sh = (st & 7) * 8;
                const u64 x0 = sb64[w], x1 = sb64[w + 1], x2 = sb64[w + 2];
                u64 b0 = sh ? (x0 >> sh) | (x1 << (64 - sh)) : x0;
                u64 b1 = sh ? (x1 >> sh) | (x2 << (64 - sh)) : x1;
                if (len < 8) {
                    b0 &= (1ull << (8 * len)) - 1;
                    b1 = 0;
                } else if (len < 16) {
                    b1 &= (1ull << (8 * (len - 8))) - 1;
                }
                return Key128{(b0 >> 60) | (b1 << 4), (b0 & ((1ull << 60) - 1)) | ((u64)len << 60)};
            };
            for (u32 q = tid; q < cntq; q += kParseThreads) {
                const u32 st = sP[q];
                const u64 en = phrase_end(q);
                const u64 len = en - st;
                if (len > (u64)kLongLen) {  // a whole warp takes it below
                    defer_long(q);
                    continue;
                }
                u32 slot = ~0u;
                int free_h = -1;
                if (len <= 7 && en <= (u64)ns) {
                    const u64 key = short_key(st, (u32)len);
                    u32 h = (u32)((key * 0x9E3779B97F4A7C15ull) >> (64 - kCacheBits));
                    for (int probe = 0; probe < kCacheProbes; probe++) {
                        const u64 k = ckey[h];
                        if (k == key) {
                            slot = cval[h];
                            break;
                        }
                        if (k == kEmpty) {
                            free_h = (int)h;
                            break;
                        }
                        h = (h + 1) & (kCacheSlots - 1);
                    }
                }
                if (slot == ~0u) {
                    bool ok = true;
                    const Key128 key = (len <= (u64)kInlineMax && en <= (u64)ns) ? byte_key(st, (u32)len) : make_key(st, en, &ok);
                    if (ok) {
                        const u32 m = atomicAdd(&s_nmiss, 1u);
                        if (m < (u32)kMissCap) {
                            sMissKey[m] = key;
                            sMissOk[m] = (okey0 + q) | ((u64)(free_h + 1) << kOkeyBits);
                            sMissPs[m] = pb0 + q;
                            continue;
                        }
                        bool claimed;  // queue full: at once (no cache entry)
                        slot = lookup_key(key, okey0 + q, &claimed);
                        if (claimed) claim_single(slot, len);
                    }
                }
                __stcs(a.P_slot + pb0 + q, slot);
            }
            __syncthreads();
            const u32 nq = s_nmiss;
            if (nq >= min(a.miss_flush ? a.miss_flush : (u32)kMissFlushDefault, (u32)kMissCap) ||
                last) {
                const u32 nm = min(nq, (u32)kMissCap);
                for (u32 i0 = 0; i0 < nm; i0 += kParseThreads) {  // whole warps take each step
                    const u32 i = i0 + tid;
                    bool claimed = false;
                    u32 slot = ~0u;
                    u64 len = 0;
                    if (i < nm) {
                        const Key128 key = sMissKey[i];
                        const u64 meta = sMissOk[i];
                        const u64 okey = meta & ((1ull << kOkeyBits) - 1);
                        const int free_h = (int)(meta >> kOkeyBits) - 1;
                        len = key_len(key);
                        slot = lookup_key(key, okey, &claimed);
                        if (free_h >= 0 && slot != ~0u && !(slot & kResidentBit)) {
                            // inline byte key of length <= 7 -> the cache's packed form
                            const u64 ck = (len << 56) | (key.hi & ((1ull << (8 * len)) - 1));
                            const u64 old = atomicCAS((unsigned long long*)&ckey[free_h], (unsigned long long)kEmpty,
                                                      (unsigned long long)ck);
                            if (old == kEmpty) cval[free_h] = slot;
                        }
                        __stcs(a.P_slot + sMissPs[i], slot);
                    }
                    claim_warp(claimed, slot, len);
                }
                __syncthreads();
                if (tid == 0) s_nmiss = 0;
            }
        } else {
            for (u32 q0 = 0; q0 < cntq; q0 += kParseThreads) {  // whole warps take each step
                const u32 q = q0 + tid;
                bool claimed = false;
                u32 slot = ~0u;
                u64 len = 0;
                if (q < cntq) {
                    const u64 st = sP[q], en = phrase_end(q);
                    len = en - st;
                    if (len > (u64)kLongLen) {  // a whole warp takes it below
                        defer_long(q);
                        len = 0;
                    } else {
                        slot = lookup(q, st, en, &claimed);
                        __stcs(a.P_slot + pb0 + q, slot);
                    }
                }
                claim_warp(claimed, slot, len);
            }
        }
        __syncthreads();

        // 4b. long phrases, one warp each: the fingerprint polynomial H
        //     (Eq. fast_hash) and the content comparisons of a hashed key are
        //     spread over the warp's lanes
        const u32 nlong = s_nlong;
        for (u32 i = warp; i < nlong; i += kParseThreads / 32) {
            const u32 q = sLong[i];
            const u64 st = sP[q], en = phrase_end(q), len = en - st;
            const u64 pos = t0 + st;  // the phrase's position in S
            u32 slot = ~0u;
            bool claimed = false;
            if (len > kMaxPhraseLen) {
                if (lane == 0) set_error(a.ds, kErrPhraseLong);
            } else {
                u64 H;
                if constexpr (kByte) {
                    H = warp_poly61([&](u64 j) -> u64 { return fp((unsigned char)sym(st + j)); }, len, a.lh.c);
                } else {
                    H = warp_poly61([&](u64 j) -> u64 { return __ldg(a.Sf + pos + j); }, len, a.lh.c);
                }
                const Key128 key = key_hashed(H, len, pos);
                u64 r = ~0ull;
                if (rt.cap)
                    r = table_find_warp(rt, key, [&](u64 rank) {
                        const u64 o = a.rrhs_off[rank];
                        return warp_equal([&](u64 j) { return (u32)S[pos + j]; },
                                          [&](u64 j) { return a.rrhs[o + j]; }, len);
                    });
                if (r != ~0ull) {
                    slot = kResidentBit | (u32)r;
                } else {
                    slot = (u32)table_claim_or_find_warp(bt, key, okey0 + q, [&](u64 ref) {
                        return warp_equal([&](u64 j) { return S[ref + j]; }, [&](u64 j) { return S[pos + j]; }, len);
                    }, &claimed, a.ds);
                }
            }
            if (lane == 0) {
                __stcs(a.P_slot + pb0 + q, slot);
                if (claimed) claim_single(slot, len);
            }
        }
        if (nlong) {
            __syncthreads();
            if (tid == 0) s_nlong = 0;
            __syncthreads();
        }

        // 5. outputs: phrase slots (from pb0 on), the tile's phrase count, and
        //    the order key of the first phrase of every string starting here
        if (tid == 0) a.tile_cnt[tile] = cntq;
        if (warp == 0) {
            for (u32 jj = j0 + lane;; jj += 32) {
                const u64 s = (jj == j0 + lane) ? s_first : (jj < kact) ? __ldg(a.soff + jj) : ~0ull;
                if (s >= t0 && s < t_end) {
                    const int x = (int)(s - t0);
                    a.string_first[jj] = okey0 + swp[x >> 5] + __popc(sbits[x >> 5] & ((1u << (x & 31)) - 1u));
                }
                if (__shfl_sync(0xffffffffu, (jj < kact && s < t_end) ? 1u : 0u, 31) == 0) break;
            }
        }
        // 6. the block's new entries join the round's claim list when the
        //    buffer is half full, and after the block's last tile
        const u32 ncl = s_nclaim;
        constexpr u32 kFlushAt = kByte ? (u32)kClaimBuf / 2 : (u32)(kClaimBuf - TP);
        static_assert(kByte || kClaimBufR >= TP, "a rank-round tile never overflows the buffer");
        if (ncl >= kFlushAt || last) {
            const u32 nb = min(ncl, (u32)kClaimBuf);
            if (tid == 0 && ncl) {
                const u64 base = atomicAdd(&a.ds->claims, (u64)nb);
                s_claim_base = base;
                atomicAdd(&a.ds->claim_len, s_claim_len);
                if (base + nb > a.claim_limit) atomicExch(&a.ds->overflow, 1u);
            }
            __syncthreads();
            if (nb) {
                const u64 base = s_claim_base;
                for (u32 x = tid; x < nb; x += kParseThreads)
                    if (base + x < bt.cap) a.claims[base + x] = sClaim[x];
            }
            __syncthreads();
            if (tid == 0) {
                s_nclaim = 0;
                s_claim_len = 0;
            }
        }
        __syncthreads();
    }
    // claims still buffered: a block whose last logical tiles were empty
    // (striped order) did not flush after its last tile
    __syncthreads();
    const u32 ncl = s_nclaim;
    if (ncl) {
        const u32 nb = min(ncl, (u32)kClaimBuf);
        if (tid == 0) {
            const u64 base = atomicAdd(&a.ds->claims, (u64)nb);
            s_claim_base = base;
            atomicAdd(&a.ds->claim_len, s_claim_len);
            if (base + nb > a.claim_limit) atomicExch(&a.ds->overflow, 1u);
        }
        __syncthreads();
        const u64 base = s_claim_base;
        for (u32 x = tid; x < nb; x += kParseThreads)
            if (base + x < bt.cap) a.claims[base + x] = sClaim[x];
    }
}

// Per parse tile: the string that holds its first position.
__device__ __forceinline__ void body_tile_strings(const RoundArgs& a, u64 tiles) {
    pdl_wait();
    const u64 n = round_n(a);
    const u32 k = round_k(a);
    const u64 nt = (n + a.tp - 1) / a.tp;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.d_tiles = nt;
        if (a.ds_prev && (vload(&a.ds_prev->error) != 0 || vload(&a.ds_prev->overflow) != 0))
            set_error(a.ds, kErrHalted);
        else if (nt > tiles)
            set_error(a.ds, kErrCapacity);
    }
    if (round_halted(a)) return;
    tiles = min(tiles, nt);
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < tiles; t += (u64)gridDim.x * blockDim.x)
        a.tile_str[t] = string_of(a.soff, k, t * (u64)a.tp);
    // bitmap of string starts (and of n), zeroed by the host
    for (u64 j = blockIdx.x * (u64)blockDim.x + threadIdx.x; j <= k; j += (u64)gridDim.x * blockDim.x) {
        const u64 s0 = __ldg(a.soff + j);
        if ((s0 >> 5) < a.sbm_words) atomicOr(a.sbm + (s0 >> 5), 1u << (s0 & 31));
    }
}

// --------------------------------------------------------------------------
// k_strings: per-string phrase ranges, retirement, next offsets (one block)
// --------------------------------------------------------------------------

__device__ __forceinline__ void body_strings(const RoundArgs& a) {
    pdl_wait();
    if (round_halted(a)) return;
    const u64 P = *a.total;
    const u32 k = round_k(a);
    u64 carry = 0;
    for (u32 j0 = 0; j0 < k; j0 += blockDim.x) {
        const u32 j = j0 + threadIdx.x;
        u64 first = 0, nextf = 0;
        bool retire = false;
        if (j < k) {
            auto index_of = [&](u64 ok) { return a.tile_pfx[ok / a.tp] + ok % a.tp; };
            first = index_of(a.string_first[j]);
            nextf = (j + 1 < k) ? index_of(a.string_first[j + 1]) : P;
            retire = (nextf - first == 1);
        }
        u64 tot;
        const u64 rb = block_excl_scan(retire ? 1ull : 0ull, tot) + carry;
        if (j < k) {
            if (retire) {
                a.R_phr[rb] = first;
                a.R_sid[rb] = a.sid[j];
            } else {
                a.soff_next[j - rb] = first - rb;
                a.sid_next[j - rb] = a.sid[j];
            }
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        a.soff_next[k - carry] = P - carry;
        a.rc->phrases = P;
        a.rc->retired = carry;
        a.rc->k_next = k - carry;
        a.rc->n_next = P - carry;
    }
}

// --------------------------------------------------------------------------
// first-occurrence naming over the claimed entries
// --------------------------------------------------------------------------

// Mark the first occurrence of every new phrase in a bitmap over phrase indices.
// Number of new rules of the round, bounded by the naming arrays.
__device__ __forceinline__ u64 round_gnew(const RoundArgs& a) {
    const u64 g = *a.d_gnew;
    if (g > a.g_alloc) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_error(a.ds, kErrCapacity);
        return a.g_alloc;
    }
    return g;
}

__device__ __forceinline__ void body_mark(const RoundArgs& a) {
    pdl_wait();
    if (round_halted(a)) return;
    const u64 g_new = round_gnew(a);
    const u64 keys = a.tiles_bound * (u64)a.tp;  // order keys the bitmap covers
    Key128* mkey = (Key128*)a.mkey;
    for (u64 c = blockIdx.x * (u64)blockDim.x + threadIdx.x; c < g_new; c += (u64)gridDim.x * blockDim.x) {
        const u32 s = a.claims[c];
        u64 m = ~0ull;
        Key128 key{0, 0};
        if (s < a.tab_cap) {  // the slot's key and value (one sector), kept in claim order for k_rank
            const Slot* sl = (const Slot*)a.tab + s;
            key = sl->key;
            m = sl->val;
        }
        mkey[c] = key;
        a.mval[c] = m;
        if (m >= keys) {
            set_error(a.ds, kErrCapacity);
            continue;
        }
        atomicOr(a.first_bits + (m >> 5), 1u << (m & 31));
    }
}

constexpr int kPopThreads = 256;
constexpr int kPopItems = 16;
constexpr int kPopTile = kPopThreads * kPopItems;

// Exclusive prefix of the popcounts of the bitmap words (single pass).
__global__ void __launch_bounds__(kPopThreads) k_popscan(const RoundArgs a, u64 nw) {
    pdl_wait();
    const u64 tile = dynamic_tile(a.ctr, a.ctr_base);
    nw = min(nw, *a.d_tiles * (u64)(a.tp / 32));
    if (tile > 0 && tile * (u64)kPopTile >= nw) return;  // beyond the count read on the device
    const u64 w0 = tile * (u64)kPopTile + (u64)threadIdx.x * kPopItems;
    static_assert(kPopItems % 4 == 0, "16-byte words");
    // a thread's words start at a multiple of 64 bytes of the arrays
    const bool full = w0 + kPopItems <= nw && ((reinterpret_cast<unsigned long long>(a.first_bits) |
                                                 reinterpret_cast<unsigned long long>(a.first_prefix)) & 15) == 0;
    u32 c[kPopItems];
    if (full) {
#pragma unroll
        for (int q = 0; q < kPopItems / 4; q++) {
            const uint4 x = reinterpret_cast<const uint4*>(a.first_bits + w0)[q];
            c[4 * q] = __popc(x.x), c[4 * q + 1] = __popc(x.y), c[4 * q + 2] = __popc(x.z), c[4 * q + 3] = __popc(x.w);
        }
    } else {
#pragma unroll
        for (int it = 0; it < kPopItems; it++) c[it] = (w0 + it < nw) ? (u32)__popc(a.first_bits[w0 + it]) : 0u;
    }
    u64 sum = 0;
#pragma unroll
    for (int it = 0; it < kPopItems; it++) sum += c[it];
    u64 tot;
    u64 e = block_excl_scan(sum, tot);
    u64 agg[1] = {tot}, excl[1];
    block_lookback<1>((LBSlot<1>*)a.lb1, tile, a.epoch, agg, excl, a.ds);
    e += excl[0];
    u32 o[kPopItems];
#pragma unroll
    for (int it = 0; it < kPopItems; it++) {
        o[it] = (u32)e;
        e += c[it];
    }
    if (full) {
        uint4* dst = reinterpret_cast<uint4*>(a.first_prefix + w0);
#pragma unroll
        for (int q = 0; q < kPopItems / 4; q++) dst[q] = make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    } else {
#pragma unroll
        for (int it = 0; it < kPopItems; it++)
            if (w0 + it < nw) a.first_prefix[w0 + it] = o[it];
    }
}

// Rank of every new phrase: the marks before its first occurrence.
__device__ __forceinline__ void body_rank(const RoundArgs& a) {
    pdl_wait();
    if (round_halted(a)) return;
    const u64 g_new = round_gnew(a);
    const Key128* mkey = (const Key128*)a.mkey;
    Key128* rkey = (Key128*)a.rkey;
    for (u64 c = blockIdx.x * (u64)blockDim.x + threadIdx.x; c < g_new; c += (u64)gridDim.x * blockDim.x) {
        const u32 s = a.claims[c];
        const u64 m = a.mval[c];  // k_mark's copy of the slot, in claim order
        if (m >= a.tiles_bound * (u64)a.tp) continue;  // k_mark flagged it
        const Key128 key = mkey[c];
        const u32 w = (u32)(m >> 5);
        const u64 r = a.first_prefix[w] + __popc(a.first_bits[w] & ((1u << (m & 31)) - 1u));
        if (r >= g_new) { set_error(a.ds, kErrCapacity); continue; }
        a.slot_r[r] = s;
        a.len_r[r] = (u32)key_len(key);
        rkey[r] = key;
    }
}

// The new rules of level i in rank order: right-hand side, offsets and F^i
// (Eq. fast_hash over F^{i-1}).  When the grammar keeps a table of its rules,
// the new rules enter it.
template <typename T>
__device__ __forceinline__ void body_rules(const RoundArgs& a) {
    pdl_wait();
    const T* S = (const T*)a.S;
    const ContentTable rw{(Slot*)a.rtab_w, a.rtab_w_cap};
    if (round_halted(a)) return;
    const u64 g_new = round_gnew(a);
    const u64 G_new = *a.d_Gnew;
    if (a.g_base + g_new > a.cap_g || a.G_base + G_new > a.cap_G) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_error(a.ds, kErrCapacity);
        return;
    }
    // whole warps step through the ranks, so that a warp can take its long
    // rules (more than kLongLen symbols) together after its short ones
    const u32 lane = threadIdx.x & 31;
    auto finish_rule = [&](u32 slot, const Key128& k, u64 len, bool hashed, u64 rank, u64 H) {
        const u32 fpv = finish_hash(a.lh, H);
        a.F[rank] = fpv;
        a.rv[slot] = ((u64)fpv << 32) | rank;  // for the rewrite: rank and fingerprint, dense by slot
        if (rw.cap) table_put(rw, hashed ? key_hashed(H, len, rank) : k, rank, a.ds);
    };
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 r0 = blockIdx.x * (u64)blockDim.x + (threadIdx.x & ~31u); r0 < g_new; r0 += stride) {
        const u64 r = r0 + lane;
        bool longr = false;
        if (r < g_new) {
            const u32 slot = a.slot_r[r];
            if (slot >= a.tab_cap) {
                set_error(a.ds, kErrCapacity);
            } else {
                const Key128 k = ((const Key128*)a.rkey)[r];  // the rule's key, in rank order (k_rank)
                const u64 len = key_len(k);
                const bool hashed = key_is_hashed(k);
                const u64 off = a.G_base + a.xlen[r];
                const u64 rank = a.g_base + r;
                a.rhs_off[rank] = off;
                if (len > (u64)kLongLen) {
                    longr = true;
                } else {
                    auto get = [&](u64 j) -> u32 { return hashed ? (u32)S[k.lo + j] : key_sym(k, j, a.sym_w); };
                    u64 H = 0;
                    for (u64 j = len; j-- > 0;) {
                        const u32 v = get(j);
                        a.rhs[off + j] = v;
                        H = addmod61(mulmod61(H, a.lh.c), (u64)__ldg(a.Fprev + v));
                    }
                    finish_rule(slot, k, len, hashed, rank, H);
                }
            }
            if (r == 0) a.rhs_off[a.g_base + g_new] = a.G_base + G_new;
        }
        // long rules (hashed keys: the content is read at the first occurrence
        // k.lo), one at a time by the whole warp
        unsigned m = __ballot_sync(0xffffffffu, longr);
        while (m) {
            const u64 rr = r0 + (u64)(__ffs(m) - 1);
            m &= m - 1;
            const u32 slot = a.slot_r[rr];
            const Key128 k = ((const Key128*)a.rkey)[rr];
            const u64 len = key_len(k);
            const u64 off = a.G_base + a.xlen[rr];
            const u64 H = warp_poly61([&](u64 j) -> u64 {
                const u32 v = (u32)S[k.lo + j];
                a.rhs[off + j] = v;
                return __ldg(a.Fprev + v);
            }, len, a.lh.c);
            if (lane == 0) finish_rule(slot, k, len, true, a.g_base + rr, H);
        }
    }
}

// --------------------------------------------------------------------------
// k_rewrite: T^{i+1} and retired strings
// --------------------------------------------------------------------------

// Phrases a thread of k_rewrite reads at once: many when the per-slot array
// it gathers from is small enough to stay in L2 (the rewrite then streams, and
// more reads in flight bring it closer to DRAM bandwidth), few when that array
// is far beyond L2 (random DRAM sectors bound it, and fewer registers keep
// more warps resident).
constexpr int kRwUnrollStream = 16, kRwUnrollGather = 4;

// T^{i+1}[p] = rank of phrase p and f^{i+1}[p] = its fingerprint F^i[rank]
// (so that the next round reads fingerprints without gathers).  Strings that
// became one phrase take their C entry instead.  The (fingerprint, rank) pair
// of a slot comes from the dense array k_rules wrote (read-only here: small
// and cached in L1 in early rounds, in L2 after its writes later on).
template <int kRwUnroll>
__device__ __forceinline__ void body_rewrite(const RoundArgs& a, u64 ntiles) {
    pdl_wait();
    if (round_halted(a)) return;
    const u64 nr = a.rc->retired;
    ntiles = min(ntiles, *a.d_tiles);
    // ranks of the level after this round (never past its arrays)
    const u64 g_total = min(a.g_base + *a.d_gnew, a.cap_g);
    const u64* __restrict__ rv = a.rv;
    // one tile per warp: the tile's header reads and its first phrase reads
    // of every warp of the SM are in flight together
    const u32 lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    const u32 stripes = a.level > 1 ? a.stripes : 1u;
    const u64 nlog = stripe_tiles(ntiles, stripes);
    for (u64 lt = (u64)blockIdx.x * warps + (threadIdx.x >> 5); lt < nlog; lt += (u64)gridDim.x * warps) {
        const u64 t = stripe_tile(lt, ntiles, stripes);
        if (t >= ntiles) continue;
        const u32 cnt = a.tile_cnt[t];
        const u64 pbase = a.tile_pfx[t];
        const u32* ps = a.P_slot + pslot_base(t, a.tile_str[t], a.tp);
        // kRwUnroll phrases per thread at a time: their reads are issued together
        for (u32 q0 = lane; q0 < cnt; q0 += kRwUnroll * 32) {
            u32 s[kRwUnroll];
            u64 v[kRwUnroll];
#pragma unroll
            for (int u = 0; u < kRwUnroll; u++) {
                const u32 q = q0 + (u32)u * 32;
                s[u] = q < cnt ? __ldcs(ps + q) : ~0u;
            }
#pragma unroll
            for (int u = 0; u < kRwUnroll; u++) {
                if (s[u] == ~0u) {
                    v[u] = 0;  // no phrase, or the round's table overflowed
                } else if (s[u] & kResidentBit) {
                    const u32 r = s[u] & ~kResidentBit;
                    v[u] = ((u64)__ldg(a.F + r) << 32) | r;
                } else {
                    v[u] = __ldg(rv + s[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < kRwUnroll; u++) {
                const u32 q = q0 + (u32)u * 32;
                if (q >= cnt) continue;
                u32 rr = (u32)v[u];
                if (rr >= g_total) {  // an entry that got no rank: only after a capacity error
                    set_error(a.ds, kErrCapacity);
                    rr = 0;
                }
                const u64 p = pbase + q;
                u64 out = p;
                if (nr != 0) {
                    u64 lo = 0, hi = nr;  // first index with R_phr >= p
                    while (lo < hi) {
                        const u64 mid = (lo + hi) >> 1;
                        if (a.R_phr[mid] < p) lo = mid + 1; else hi = mid;
                    }
                    if (lo < nr && a.R_phr[lo] == p) {
                        a.c_level[a.R_sid[lo]] = a.level;
                        a.c_rank[a.R_sid[lo]] = rr;
                        continue;
                    }
                    out = p - lo;
                }
                if (out >= a.T_cap) {
                    set_error(a.ds, kErrCapacity);
                    continue;
                }
                __stcs(a.Tnext + out, rr);
                __stcs(a.Fnext + out, (u32)(v[u] >> 32));
            }
        }
    }
}

// --------------------------------------------------------------------------
// k_resident_build: table over existing rules of a level
// --------------------------------------------------------------------------

// Rules r0 .. r0+cnt-1 of a level enter its table (values: ranks).
template <bool kByte>
__global__ void k_resident_build(const u32* __restrict__ rhs, const u64* __restrict__ rhs_off, u64 r0, u64 cnt,
                                 const u32* __restrict__ Fprev, LevelHash lh, ContentTable t, DevStatus* ds) {
    pdl_wait();
    for (u64 x = blockIdx.x * (u64)blockDim.x + threadIdx.x; x < cnt; x += (u64)gridDim.x * blockDim.x) {
        const u64 r = r0 + x;
        const u64 s = rhs_off[r], e = rhs_off[r + 1];
        u64 H = 0;
        for (u64 y = e; y-- > s;) H = addmod61(mulmod61(H, lh.c), (u64)__ldg(Fprev + rhs[y]));
        const Key128 k = rule_key([&](u64 j) { return rhs[s + j]; }, e - s, kByte ? 8 : kRankBits, H, r);
        table_put(t, k, r, ds);
    }
}

// --------------------------------------------------------------------------
// round 0 helpers: strings of length one, and gathering the active strings
// --------------------------------------------------------------------------

__global__ void k_level0(const unsigned char* __restrict__ data, const u64* __restrict__ pos,
                         const u32* __restrict__ ids, u32 cnt, u32* c_level, u32* c_rank) {
    pdl_wait();
    const u32 x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < cnt) {
        c_level[ids[x]] = 0;
        c_rank[ids[x]] = data[pos[x]];
    }
}

__global__ void k_gather_strings(const unsigned char* __restrict__ data, const u64* __restrict__ src_off,
                                 const u64* __restrict__ dst_off, u32 k, unsigned char* __restrict__ out) {
    pdl_wait();
    for (u32 j = blockIdx.x; j < k; j += gridDim.x) {
        const u64 s = src_off[j], d = dst_off[j], len = dst_off[j + 1] - dst_off[j];
        for (u64 x = threadIdx.x; x < len; x += blockDim.x) out[d + x] = data[s + x];
    }
}

// --------------------------------------------------------------------------
// host launchers
// --------------------------------------------------------------------------

// --------------------------------------------------------------------------
// the round's kernels, and the short rounds' cooperative kernels
// --------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(kBrkThreads) k_breaks(const RoundArgs a, u64 nblocks) { body_breaks<T>(a, nblocks); }
template <typename T, int TP>
__global__ void __launch_bounds__(kParseThreads, sizeof(T) == 1 ? 5 : 4) k_parse(const RoundArgs a, u64 ntiles) {
    body_parse<T, TP>(a, ntiles);
}
__global__ void k_tile_strings(const RoundArgs a, u64 tiles) { body_tile_strings(a, tiles); }
__global__ void __launch_bounds__(1024) k_strings(const RoundArgs a) { body_strings(a); }
__global__ void k_mark(const RoundArgs a) { body_mark(a); }
__global__ void k_rank(const RoundArgs a) { body_rank(a); }
template <typename T>
__global__ void k_rules(const RoundArgs a) { body_rules<T>(a); }
template <int kRwUnroll>
__global__ void __launch_bounds__(256) k_rewrite(const RoundArgs a, u64 ntiles) { body_rewrite<kRwUnroll>(a, ntiles); }

// Exclusive prefix of in[0 .. n) (n: the smaller of the bound and *n_dev when
// given) into out, the sum into totals[0] and 0 into totals[1] (what k_scan2
// gives for one column), by one block of kSmallThreads threads.
constexpr int kSmallThreads = 256;
constexpr int kSmallItems = 16;
template <typename Get>
__device__ void block_scan_small(Get get, u64 n, const u64* n_dev, u64* out64, u32* out32, u64* totals) {
    if (n_dev != nullptr) n = min(*n_dev, n);
    u64 carry = 0;
    for (u64 base = 0; base < n; base += (u64)kSmallThreads * kSmallItems) {
        const u64 p0 = base + (u64)threadIdx.x * kSmallItems;
        u32 v[kSmallItems];
        u64 sum = 0;
#pragma unroll
        for (int i = 0; i < kSmallItems; i++) {
            v[i] = p0 + i < n ? get(p0 + i) : 0u;
            sum += v[i];
        }
        u64 tot;
        u64 e = block_excl_scan(sum, tot) + carry;
#pragma unroll
        for (int i = 0; i < kSmallItems; i++) {
            if (p0 + i < n) {
                if (out64) out64[p0 + i] = e;
                if (out32) out32[p0 + i] = (u32)e;
            }
            e += v[i];
        }
        carry += tot;
    }
    if (threadIdx.x == 0 && totals != nullptr) {
        totals[0] = carry;
        totals[1] = 0;
    }
    __syncthreads();
}

// Barrier over the grid of a cooperative launch: the k-th barrier of a launch
// waits until the round's counter has reached base + k * gridDim.x (every
// block arrived).  Bounded: after kSpinLimit polls the round fails with
// kErrTimeout and the kernel's later steps return at once.
__device__ void grid_barrier(u64* ctr, u64 target, DevStatus* ds) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1ull);
        u64 it = 0;
        u32 backoff = 32;
        while (true) {
            u64 v;
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctr) : "memory");
            if (v >= target) break;
            if (++it > kSpinLimit) {
                set_error(ds, kErrTimeout);
                break;
            }
            __nanosleep(backoff);
            if (backoff < 256) backoff <<= 1;
        }
        __threadfence();
    }
    __syncthreads();
}

// A short round's parse in one cooperative launch instead of five: tile
// strings, breaks, k_parse over the tiles (grid-stride, like the launches),
// then block 0 scans the tiles' phrase counts and runs the per-string pass.
// Grid barriers separate the steps.  Same buffers and results as the launches.
template <typename T>
__global__ void __launch_bounds__(kSmallThreads) k_parse_small(const RoundArgs a, u64 tiles, u64 nsteps,
                                                                u64 bar_base) {
    static_assert(kSmallThreads == kParseThreads && kSmallThreads == kBrkThreads, "one block shape");
    const u64 g = gridDim.x;
    body_tile_strings(a, tiles);
    grid_barrier(a.ctr, bar_base + g, a.ds);
    body_breaks<T>(a, nsteps);
    grid_barrier(a.ctr, bar_base + 2 * g, a.ds);
    body_parse<T, kTPMin>(a, tiles);
    grid_barrier(a.ctr, bar_base + 3 * g, a.ds);
    if (blockIdx.x == 0) {
        block_scan_small([&](u64 i) { return a.tile_cnt[i]; }, tiles, a.d_tiles, a.tile_pfx, nullptr, a.total);
        body_strings(a);
    }
}

// A short round's naming and rewrite in one cooperative launch instead of
// six: marks, (block 0) the prefix of the marks' popcounts, ranks, (block 0)
// the scan of the rule lengths, rules and the rewrite.
template <typename T>
__global__ void __launch_bounds__(kSmallThreads) k_naming_small(const RoundArgs a, u64 nw, u64 g_bound,
                                                                 u64 bar_base) {
    const u64 g = gridDim.x;
    body_mark(a);
    grid_barrier(a.ctr, bar_base + g, a.ds);
    if (blockIdx.x == 0)
        block_scan_small([&](u64 w) { return (u32)__popc(a.first_bits[w]); },
                         min(nw, *a.d_tiles * (u64)(a.tp / 32)), nullptr, nullptr, a.first_prefix, nullptr);
    grid_barrier(a.ctr, bar_base + 2 * g, a.ds);
    body_rank(a);
    grid_barrier(a.ctr, bar_base + 3 * g, a.ds);
    if (blockIdx.x == 0)
        block_scan_small([&](u64 i) { return a.len_r[i]; }, g_bound, a.d_gnew, a.xlen, nullptr, a.total + 1);
    grid_barrier(a.ctr, bar_base + 4 * g, a.ds);
    body_rules<T>(a);
    grid_barrier(a.ctr, bar_base + 5 * g, a.ds);
    body_rewrite<kRwUnrollGather>(a, a.tiles_bound);
}

static unsigned grid_for(u64 n, u64 cap = 152ull * 32) {
    u64 b = (n + 255) / 256;
    if (b == 0) b = 1;
    return (unsigned)(b < cap ? b : cap);
}

bool parse_tile_valid(u32 tp) { return tp == 1024 || tp == 2048 || tp == 4096; }
u64 parse_slot_entries(u64 tiles, u64 strings, u32 tp) { return tiles * (u64)(tp / 2 + 2) + strings + 1; }
u64 breaks_steps(u64 tiles, u32 tp) { return (tiles * (u64)tp + kBrkSpan - 1) / kBrkSpan + 1; }

u64 popscan_tiles_for(u64 nw) { return (nw + kPopTile - 1) / kPopTile; }

cudaError_t launch_tile_strings(const RoundArgs& a, cudaStream_t st) {
    return launch_pdl(k_tile_strings, grid_for(a.tiles_bound), 256, st, a, a.tiles_bound);
}

template <typename T, int TP>
static int parse_occupancy(int* sms_out) {
    // queried once per instantiation (thread-safe static initialisation:
    // contexts on several host threads launch at once)
    static const std::pair<int, int> occ_sms = [] {
        int dev = 0, sms = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_parse<T, TP>, kParseThreads, 0);
        return std::make_pair(occ > 0 ? occ : 1, sms);
    }();
    if (sms_out) *sms_out = occ_sms.second;
    return occ_sms.first;
}

// Persistent grid: `per_sm` blocks per SM (0 or more than fit: as many as fit).
template <typename T, int TP>
static unsigned persistent_grid(u64 tiles, u32 per_sm) {
    int sms = 0;
    const int occ = parse_occupancy<T, TP>(&sms);
    const u64 b = (per_sm == 0 || per_sm > (u32)occ) ? (u64)occ : (u64)per_sm;
    const u64 g = b * (u64)sms;
    return (unsigned)(tiles < g ? (tiles ? tiles : 1) : g);
}

// Most k_parse blocks that fit on an SM, over every tile size.
int parse_max_blocks(int sym_bytes) {
    if (sym_bytes == 1)
        return std::max({parse_occupancy<unsigned char, 1024>(nullptr), parse_occupancy<unsigned char, 2048>(nullptr),
                         parse_occupancy<unsigned char, 4096>(nullptr)});
    return std::max({parse_occupancy<u32, 1024>(nullptr), parse_occupancy<u32, 2048>(nullptr),
                     parse_occupancy<u32, 4096>(nullptr)});
}

template <typename T>
static unsigned breaks_grid(u64 blocks) {
    static const u64 cap = [] {
        int dev = 0, sms = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_breaks<T>, kBrkThreads, 0);
        return (u64)(occ > 0 ? occ : 1) * (u64)sms;
    }();
    return (unsigned)(blocks < cap ? (blocks ? blocks : 1) : cap);
}

cudaError_t launch_breaks(const RoundArgs& a, cudaStream_t st) {
    const u64 blocks = (a.tiles_bound * (u64)a.tp + kBrkSpan - 1) / kBrkSpan;
    if (a.sym_bytes == 1)
        return launch_pdl(k_breaks<unsigned char>, breaks_grid<unsigned char>(blocks), kBrkThreads, st, a, blocks);
    return launch_pdl(k_breaks<u32>, breaks_grid<u32>(blocks), kBrkThreads, st, a, blocks);
}

template <typename T, int TP>
static cudaError_t launch_parse_tp(const RoundArgs& a, cudaStream_t st) {
    const u64 tiles = a.tiles_bound;
    return launch_pdl(k_parse<T, TP>, persistent_grid<T, TP>(tiles, a.parse_blocks), kParseThreads, st, a, tiles);
}

template <typename T>
static cudaError_t launch_parse_t(const RoundArgs& a, cudaStream_t st) {
    switch (a.tp) {
        case 1024: return launch_parse_tp<T, 1024>(a, st);
        case 2048: return launch_parse_tp<T, 2048>(a, st);
        case 4096: return launch_parse_tp<T, 4096>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_parse(const RoundArgs& a, cudaStream_t st) {
    if (a.sym_bytes == 1) return launch_parse_t<unsigned char>(a, st);
    return launch_parse_t<u32>(a, st);
}

bool round_is_small(const RoundArgs& a) { return a.tp == (u32)kTPMin && a.tiles_bound <= kSmallTiles; }

// Blocks of a short round's cooperative launches: one per tile, at most one
// per SM (and never more than can be resident at once).
u32 small_round_grid(const RoundArgs& a) {
    static const int cap = [] {
        int dev = 0, sms = 0, o1 = 0, o2 = 0, o3 = 0, o4 = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_parse_small<unsigned char>, kSmallThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_parse_small<u32>, kSmallThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o3, k_naming_small<unsigned char>, kSmallThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o4, k_naming_small<u32>, kSmallThreads, 0);
        // one block per SM (a cooperative launch checks that they fit)
        return (std::min({o1, o2, o3, o4}) >= 1 && sms > 0) ? sms : 1;
    }();
    return (u32)std::min<u64>((u64)cap, std::max<u64>(1, a.tiles_bound));
}

cudaError_t launch_parse_small(const RoundArgs& a, u64 bar_base, cudaStream_t st) {
    const u64 nsteps = (a.tiles_bound * (u64)a.tp + kBrkSpan - 1) / kBrkSpan;
    const u32 g = small_round_grid(a);
    if (a.sym_bytes == 1)
        return launch_coop(k_parse_small<unsigned char>, g, kSmallThreads, st, a, a.tiles_bound, nsteps, bar_base);
    return launch_coop(k_parse_small<u32>, g, kSmallThreads, st, a, a.tiles_bound, nsteps, bar_base);
}

cudaError_t launch_naming_small(const RoundArgs& a, u64 nw, u64 g_bound, u64 bar_base, cudaStream_t st) {
    const u32 g = small_round_grid(a);
    if (a.sym_bytes == 1)
        return launch_coop(k_naming_small<unsigned char>, g, kSmallThreads, st, a, nw, g_bound, bar_base);
    return launch_coop(k_naming_small<u32>, g, kSmallThreads, st, a, nw, g_bound, bar_base);
}

cudaError_t launch_strings(const RoundArgs& a, cudaStream_t st) {
    return launch_pdl(k_strings, 1, 1024, st, a);
}

cudaError_t launch_mark(const RoundArgs& a, u64 g_grid, cudaStream_t st) {
    return launch_pdl(k_mark, grid_for(g_grid), 256, st, a);
}

cudaError_t launch_popscan(const RoundArgs& a, u64 nw_bound, cudaStream_t st) {
    u64 tiles = popscan_tiles_for(nw_bound);
    if (tiles == 0) tiles = 1;
    return launch_pdl(k_popscan, (unsigned)tiles, kPopThreads, st, a, nw_bound);
}

cudaError_t launch_rank(const RoundArgs& a, u64 g_grid, cudaStream_t st) {
    return launch_pdl(k_rank, grid_for(g_grid), 256, st, a);
}

cudaError_t launch_rules(const RoundArgs& a, u64 g_grid, cudaStream_t st) {
    if (a.sym_bytes == 1) return launch_pdl(k_rules<unsigned char>, grid_for(g_grid), 256, st, a);
    return launch_pdl(k_rules<u32>, grid_for(g_grid), 256, st, a);
}

cudaError_t launch_rewrite(const RoundArgs& a, cudaStream_t st) {
    const u64 tiles = a.tiles_bound;
    const u64 blocks = (tiles + 7) / 8;  // 8 warps per block, one tile each
    const u64 g = blocks < 152ull * 8 ? (blocks ? blocks : 1) : 152ull * 8;
    if ((double)a.tab_cap * sizeof(u64) <= kL2Bytes)
        return launch_pdl(k_rewrite<kRwUnrollStream>, (unsigned)g, 256, st, a, tiles);
    return launch_pdl(k_rewrite<kRwUnrollGather>, (unsigned)g, 256, st, a, tiles);
}

cudaError_t launch_level0(const unsigned char* data, const u64* pos, const u32* ids, u32 cnt, u32* c_level,
                          u32* c_rank, cudaStream_t st) {
    if (cnt == 0) return cudaSuccess;
    k_level0<<<(cnt + 255) / 256, 256, 0, st>>>(data, pos, ids, cnt, c_level, c_rank);
    return cudaGetLastError();
}

cudaError_t launch_gather_strings(const unsigned char* data, const u64* src_off, const u64* dst_off, u32 k,
                                  unsigned char* out, cudaStream_t st) {
    if (k == 0) return cudaSuccess;
    const unsigned blocks = k < 152 * 8 ? k : 152 * 8;
    k_gather_strings<<<blocks, 256, 0, st>>>(data, src_off, dst_off, k, out);
    return cudaGetLastError();
}

cudaError_t launch_resident_build(const u32* rhs, const u64* rhs_off, u64 r0, u64 cnt, bool bytes, const u32* Fprev,
                                  LevelHash lh, void* slots, u64 cap, DevStatus* ds, cudaStream_t st) {
    if (cnt == 0) return cudaSuccess;
    const ContentTable t{(Slot*)slots, cap};
    if (bytes) k_resident_build<true><<<grid_for(cnt), 256, 0, st>>>(rhs, rhs_off, r0, cnt, Fprev, lh, t, ds);
    else k_resident_build<false><<<grid_for(cnt), 256, 0, st>>>(rhs, rhs_off, r0, cnt, Fprev, lh, t, ds);
    return cudaGetLastError();
}

size_t lb1_bytes(u64 tiles) { return tiles * sizeof(LBSlot<1>); }
size_t lb2_bytes(u64 tiles) { return tiles * sizeof(LBSlot<2>); }
size_t slot_bytes() { return sizeof(Slot); }

}  // namespace lcg
