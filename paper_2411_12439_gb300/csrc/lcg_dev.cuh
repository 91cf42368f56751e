// Device-side building blocks shared by the kernels of the library:
// arithmetic modulo the Mersenne prime 2^61-1, the decoupled look-back used by
// the single-pass scans, the device status word through which bounded waits
// report failure, and the wait of programmatic dependent launch.  (The phrase
// table is in table.cuh.)
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lcg {

typedef unsigned long long u64;
typedef unsigned int u32;
typedef unsigned char u8;

// --------------------------------------------------------------------------
// arithmetic modulo p = 2^61 - 1
// --------------------------------------------------------------------------

constexpr u64 kP61 = 2305843009213693951ull;

// a * b mod p for a, b < p.  Mersenne folding: with x = a*b = x_hi 2^61 + x_lo,
// 2^61 = 1 (mod p) gives x = x_hi + x_lo (mod p); both parts are < 2^61, so
// one conditional subtraction finishes the reduction.
__device__ __forceinline__ u64 mulmod61(u64 a, u64 b) {
    u64 lo = a * b;
    u64 hi = __umul64hi(a, b);
    u64 r = (lo & kP61) + ((lo >> 61) | (hi << 3));
    return r >= kP61 ? r - kP61 : r;
}

__device__ __forceinline__ u64 addmod61(u64 a, u64 b) {  // a, b < p
    u64 r = a + b;
    return r >= kP61 ? r - kP61 : r;
}

// Level hash parameters of one level (Sec. 3.2).
struct LevelHash {
    u64 a, b, c;
    u64 mmask;  // m - 1
};

// c^e mod p (square and multiply).
__device__ __forceinline__ u64 powmod61(u64 c, u64 e) {
    u64 r = 1;
    while (e) {
        if (e & 1) r = mulmod61(r, c);
        c = mulmod61(c, c);
        e >>= 1;
    }
    return r;
}

// H = sum_{j < len} v(j) c^j mod p (the polynomial of Eq. fast_hash), by a
// whole warp: every lane calls it with the same len and c.  Lane l takes the
// terms j = l, l + 32, ...: h_l = sum_k v(32k + l) (c^32)^k by Horner over
// k, read 32 consecutive terms per warp step; then H = sum_l c^l h_l.
// Every lane returns H.  v(j) must be < p.
template <typename V>
__device__ __forceinline__ u64 warp_poly61(V v, u64 len, u64 c) {
    const u32 lane = threadIdx.x & 31;
    const u64 c32 = powmod61(c, 32);
    constexpr int U = 4;  // terms read before they enter the dependent chain
    u64 h = 0;
    u64 kk = (len + 31) / 32;
    while (kk > 0) {
        const int m = kk < (u64)U ? (int)kk : U;
        u64 x[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const u64 j = 32 * (kk - 1 - (u64)u) + lane;
            x[u] = (u < m && j < len) ? (u64)v(j) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < U; u++)
            if (u < m) h = addmod61(mulmod61(h, c32), x[u]);
        kk -= (u64)m;
    }
    h = mulmod61(h, powmod61(c, lane));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h = addmod61(h, __shfl_xor_sync(0xffffffffu, h, o));
    return h;
}

// a(j) == b(j) for every j < len, by a whole warp (every lane gets the answer).
template <typename A, typename B>
__device__ __forceinline__ bool warp_equal(A a, B b, u64 len) {
    const u32 lane = threadIdx.x & 31;
    constexpr int U = 8;
    for (u64 j0 = 0; j0 < len; j0 += 32 * U) {
        bool ok = true;
#pragma unroll
        for (int u = 0; u < U; u++) {
            const u64 j = j0 + 32 * (u64)u + lane;
            if (j < len) ok = ok && (a(j) == b(j));
        }
        if (!__all_sync(0xffffffffu, ok)) return false;
    }
    return true;
}

// ((a * H + b) mod p) mod m for a polynomial value H < p (Eq. fast_hash).
__device__ __forceinline__ u32 finish_hash(const LevelHash& h, u64 H) {
    return (u32)(addmod61(mulmod61(h.a, H), h.b) & h.mmask);
}

// 64-bit finaliser of MurmurHash3 (public domain): spreads a value's bits.
__device__ __forceinline__ u64 fmix64(u64 k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// --------------------------------------------------------------------------
// device status
// --------------------------------------------------------------------------

enum DevError : u32 {
    kErrNone = 0,
    kErrTimeout = 1,      // a bounded wait ran out
    kErrTableFull = 2,    // a probe sequence visited every slot
    kErrPhraseLong = 3,   // a phrase of >= 2^32 symbols
    kErrMismatch = 4,     // equal right-hand sides with different fingerprints
    kErrRankOverflow = 5, // a level with >= 2^32 rules
    kErrCapacity = 6,     // a round outgrew the buffers it was given (rounds enqueued without a sync)
    kErrHalted = 7,       // an earlier round failed; this one did no work
    kErrFormat = 8,       // a malformed VByte stream
};

struct DevStatus {
    u32 error;        // first DevError seen
    u32 overflow;     // phrase table passed its load limit (host regrows)
    u64 claims;       // slots claimed in the current table pass
    u64 claim_len;    // total length of the claimed phrases
    u64 aux[5];
};

// Kernels of a build are launched with programmatic dependent launch: a grid
// may be scheduled while the one before it drains, and waits here, before its
// first access to memory, until that grid has finished and its writes are
// visible.  (A no-op for a grid launched without the attribute.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void set_error(DevStatus* st, u32 code) {
    atomicCAS(&st->error, 0u, code);
}

__device__ __forceinline__ u32 vload(const volatile u32* p) { return *p; }
__device__ __forceinline__ u64 vload(const volatile u64* p) { return *p; }

constexpr u64 kSpinLimit = 1ull << 22;  // bounded waits: about a second at most

// Empty marker of 64-bit keys in shared-memory caches.
constexpr u64 kEmpty = ~0ull;

// --------------------------------------------------------------------------
// decoupled look-back (single-pass prefix sums over tiles in launch order)
// --------------------------------------------------------------------------
//
// Each tile publishes its aggregate, then its inclusive prefix, in an
// LBSlot.  The flag word carries the launch epoch so that slots left by an
// earlier launch read as "not yet published": no clearing between launches.
// Tiles take their index from a counter in launch order, so a tile only ever
// waits on tiles already running.

template <int NV>
struct LBSlot {
    u64 flag;  // (epoch << 2) | state, state 1 = aggregate, 2 = inclusive prefix
    u64 agg[NV];
    u64 incl[NV];
};

// Publish a tile's aggregate (thread 0).  Tile 0 publishes its inclusive
// prefix at once.
template <int NV>
__device__ __forceinline__ void lookback_publish(LBSlot<NV>* st, u64 tile, u64 epoch, const u64 (&agg)[NV]) {
    volatile LBSlot<NV>* vs = st;
#pragma unroll
    for (int v = 0; v < NV; v++) {
        vs[tile].agg[v] = agg[v];
        if (tile == 0) vs[0].incl[v] = agg[v];
    }
    __threadfence();
    vs[tile].flag = (epoch << 2) | (tile == 0 ? 2 : 1);
}

// Block-wide, after lookback_publish: wait for the predecessors, publish the
// tile's inclusive prefix and return the exclusive one in `excl` (every
// thread).  Needs blockDim.x >= 32.  On a timeout the error is set and the
// prefix is 0.
template <int NV>
__device__ void lookback_finish(LBSlot<NV>* st, u64 tile, u64 epoch, const u64 (&agg)[NV], u64 (&excl)[NV],
                                DevStatus* ds) {
    __shared__ u64 s_excl[NV];
    if (threadIdx.x < 32) {
        const u32 lane = threadIdx.x;
        volatile LBSlot<NV>* vs = st;
        u64 acc[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) acc[v] = 0;
        if (tile != 0) {
            long long base = (long long)tile - 1;
            bool failed = false;
            while (true) {
                const long long idx = base - (long long)lane;
                u32 state = 2;  // virtual tiles before 0: inclusive, value 0
                if (idx >= 0) {
                    u64 it = 0;
                    u32 backoff = 16;
                    while (true) {
                        const u64 f = vs[idx].flag;
                        if ((f >> 2) == epoch && (f & 3) != 0) { state = (u32)(f & 3); break; }
                        if (++it > kSpinLimit || vload(&ds->error) != 0) { state = 0; break; }
                        // back off so that waiting warps leave issue slots to working
                        // ones, but not so far that a ready predecessor waits long
                        __nanosleep(backoff);
                        if (backoff < 256) backoff <<= 1;
                    }
                }
                if (__any_sync(0xffffffffu, state == 0)) { failed = true; break; }
                const u32 incl_mask = __ballot_sync(0xffffffffu, state == 2);
                __threadfence();
                const int first = incl_mask ? __ffs(incl_mask) - 1 : 31;
#pragma unroll
                for (int v = 0; v < NV; v++) {
                    u64 val = 0;
                    if (idx >= 0 && (int)lane <= first) val = (state == 2) ? vs[idx].incl[v] : vs[idx].agg[v];
                    for (int o = 16; o > 0; o >>= 1) val += __shfl_down_sync(0xffffffffu, val, o);
                    acc[v] += val;
                }
                if (incl_mask) break;
                base -= 32;
            }
            if (failed) {
                if (lane == 0) set_error(ds, kErrTimeout);
#pragma unroll
                for (int v = 0; v < NV; v++) acc[v] = 0;
            }
            if (lane == 0) {
#pragma unroll
                for (int v = 0; v < NV; v++) vs[tile].incl[v] = acc[v] + agg[v];
                __threadfence();
                vs[tile].flag = (epoch << 2) | 2;
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int v = 0; v < NV; v++) s_excl[v] = acc[v];
        }
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < NV; v++) excl[v] = s_excl[v];
    __syncthreads();
}

// Both steps at once: every thread passes the tile's aggregate in `agg` (only
// thread 0's value is used) and receives the exclusive prefix in `excl`.
template <int NV>
__device__ void block_lookback(LBSlot<NV>* st, u64 tile, u64 epoch, const u64 (&agg)[NV], u64 (&excl)[NV],
                               DevStatus* ds) {
    if (threadIdx.x == 0) lookback_publish<NV>(st, tile, epoch, agg);
    lookback_finish<NV>(st, tile, epoch, agg, excl, ds);
}

// Tile index in launch order from a counter that is never reset: the host
// passes the counter's value at launch (`ctr_base`).
__device__ __forceinline__ u64 dynamic_tile(u64* ctr, u64 ctr_base) {
    __shared__ u64 s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(ctr, 1ull) - ctr_base;
    __syncthreads();
    u64 t = s_tile;
    __syncthreads();
    return t;
}

// Block-wide exclusive scan of one u64 per thread (blockDim.x a multiple of 32,
// at most 1024).  Returns the exclusive prefix; `total` gets the block sum.
__device__ __forceinline__ u64 block_excl_scan(u64 x, u64& total) {
    __shared__ u64 s_warp[32];
    __shared__ u64 s_total;
    const u32 lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    u64 incl = x;
    for (int o = 1; o < 32; o <<= 1) {
        u64 y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        u64 w = lane < nw ? s_warp[lane] : 0;
        u64 wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            u64 y = __shfl_up_sync(0xffffffffu, wi, o);
            if ((int)lane >= o) wi += y;
        }
        if (lane < nw) s_warp[lane] = wi - w;  // exclusive warp offsets
        if (lane == nw - 1) s_total = wi;
    }
    __syncthreads();
    u64 res = s_warp[wid] + incl - x;
    total = s_total;
    __syncthreads();
    return res;
}

}  // namespace lcg
