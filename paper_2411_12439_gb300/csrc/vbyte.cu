// VByte codec of the grammar's arrays (Sec. 4, resource usage: rules stored
// with VBytes instead of 32-bit cells).  A value is cut into groups of 7 bits,
// least significant group first, one group per byte; the high bit of a byte
// is set when another byte of the same value follows (the LEB128 / varint
// layout).
//
// Both directions are single-pass over tiles with a decoupled look-back:
//   k_vb_encode: a tile of 2048 values -> byte counts -> block scan ->
//     look-back gives the tile's byte offset; the tile's bytes are assembled
//     in shared memory and stored with 4-byte stores (edges byte by byte), so
//     the stream is written once, coalesced.
//   k_vb_decode: a tile of 4096 stream bytes (plus the 8 bytes before it) in
//     shared memory; every byte without the high bit ends a value, which is
//     assembled from the bytes before it; counts (and, for rule lengths, the
//     sums) are scanned across tiles by look-back and the tile's values are
//     stored coalesced.  Malformed streams (a value of more than 32 bits, a
//     stream that ends inside a value, a value outside the allowed range, a
//     different number of values) set kErrFormat; no write leaves the output.
// Rule lengths are encoded straight from the u64 offsets and decoded straight
// into them (the lengths array never exists), so an export or import of a
// level reads and writes each array once.
#include "lcg_dev.cuh"
#include "lcg_internal.h"

namespace lcg {

constexpr int kVbThreads = 256;
constexpr int kVbItems = 8;                         // values per thread (encode)
constexpr int kVbTile = kVbThreads * kVbItems;      // 2048 values
constexpr int kVbBytes = 16;                        // stream bytes per thread (decode)
constexpr int kVbDecTile = kVbThreads * kVbBytes;   // 4096 bytes
constexpr int kVbHalo = 8;                          // bytes before a decode tile

__device__ __forceinline__ u32 vb_len(u32 v) {
    return 1u + (v >= (1u << 7)) + (v >= (1u << 14)) + (v >= (1u << 21)) + (v >= (1u << 28));
}

// Value p of the column: a u32 array, or the lengths rhs_off[p+1] - rhs_off[p].
template <bool kLens>
__device__ __forceinline__ u32 vb_value(const u32* vals, const u64* offs, u64 p) {
    if (kLens) return (u32)(__ldg(offs + p + 1) - __ldg(offs + p));
    return __ldg(vals + p);
}

// --------------------------------------------------------------------------
// byte count of a column (sizes the sections of an export)
// --------------------------------------------------------------------------

template <bool kLens>
__global__ void __launch_bounds__(kVbThreads) k_vb_count(const u32* __restrict__ vals, const u64* __restrict__ offs,
                                                         u64 n, u64* __restrict__ total) {
    pdl_wait();
    u64 s = 0;
    for (u64 p = blockIdx.x * (u64)blockDim.x + threadIdx.x; p < n; p += (u64)gridDim.x * blockDim.x)
        s += vb_len(vb_value<kLens>(vals, offs, p));
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ u64 s_w[kVbThreads / 32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 t = 0;
        for (int w = 0; w < kVbThreads / 32; w++) t += s_w[w];
        if (t) atomicAdd(reinterpret_cast<unsigned long long*>(total), (unsigned long long)t);
    }
}

// --------------------------------------------------------------------------
// encode
// --------------------------------------------------------------------------

// Writes the VByte stream of the n values to out[0 ..), with `pad` zeros up
// to the next multiple of 8 bytes (the section padding), and the stream's
// length to *nbytes_out.
template <bool kLens>
__global__ void __launch_bounds__(kVbThreads) k_vb_encode(const u32* __restrict__ vals, const u64* __restrict__ offs,
                                                          u64 n, u8* __restrict__ out, u64* __restrict__ nbytes_out,
                                                          bool pad, LBSlot<2>* lb, u64 epoch, u64* ctr, u64 ctr_base,
                                                          DevStatus* ds) {
    __shared__ u8 s_out[kVbTile * 5];
    pdl_wait();
    const u64 tile = dynamic_tile(ctr, ctr_base);
    const u64 p0 = tile * (u64)kVbTile + (u64)threadIdx.x * kVbItems;
    u32 v[kVbItems];
    u32 mine = 0;
    if (!kLens && p0 + kVbItems <= n && (reinterpret_cast<uintptr_t>(vals + p0) & 15) == 0) {
        const uint4 a = __ldg(reinterpret_cast<const uint4*>(vals + p0));
        const uint4 b = __ldg(reinterpret_cast<const uint4*>(vals + p0) + 1);
        v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
    } else if (kLens) {
        u64 prev = (p0 < n) ? __ldg(offs + p0) : 0;
#pragma unroll
        for (int it = 0; it < kVbItems; it++) {
            const u64 nx = (p0 + it < n) ? __ldg(offs + p0 + it + 1) : prev;
            v[it] = (u32)(nx - prev);
            prev = nx;
        }
    } else {
#pragma unroll
        for (int it = 0; it < kVbItems; it++) v[it] = (p0 + it < n) ? __ldg(vals + p0 + it) : 0u;
    }
#pragma unroll
    for (int it = 0; it < kVbItems; it++) mine += (p0 + it < n) ? vb_len(v[it]) : 0u;
    u64 tile_bytes;
    const u64 my_off = block_excl_scan(mine, tile_bytes);
    u64 agg[2] = {tile_bytes, 0}, excl[2];
    block_lookback<2>(lb, tile, epoch, agg, excl, ds);
    // assemble the tile's bytes in shared memory
    u32 o = (u32)my_off;
#pragma unroll
    for (int it = 0; it < kVbItems; it++) {
        if (p0 + it < n) {
            u32 x = v[it];
            while (x >= 0x80u) {
                s_out[o++] = (u8)(x | 0x80u);
                x >>= 7;
            }
            s_out[o++] = (u8)x;
        }
    }
    __syncthreads();
    // store [base, base + tile_bytes): edge bytes one by one, the rest as words
    u8* dst = out + excl[0];
    const u32 tb = (u32)tile_bytes;
    const u32 head = min(tb, (u32)((4 - (reinterpret_cast<uintptr_t>(dst) & 3)) & 3));
    const u32 words = (tb - head) >> 2;
    const u32 tail0 = head + 4 * words;
    if (threadIdx.x < head) dst[threadIdx.x] = s_out[threadIdx.x];
    for (u32 t = tail0 + threadIdx.x; t < tb; t += kVbThreads) dst[t] = s_out[t];
    u32* wdst = reinterpret_cast<u32*>(dst + head);
    for (u32 w = threadIdx.x; w < words; w += kVbThreads) {
        const u32 b = head + 4 * w;
        wdst[w] = (u32)s_out[b] | ((u32)s_out[b + 1] << 8) | ((u32)s_out[b + 2] << 16) | ((u32)s_out[b + 3] << 24);
    }
    if ((tile + 1) * (u64)kVbTile >= n && threadIdx.x == 0) {
        const u64 total = excl[0] + tile_bytes;
        if (pad)
            for (u64 z = total; z & 7; z++) out[z] = 0;
        *nbytes_out = total;
    }
}

// --------------------------------------------------------------------------
// decode
// --------------------------------------------------------------------------

// The value whose last byte is sb[q]: its bytes are that byte and the
// continuation bytes right before it.  More than 5 bytes or 32 bits sets `bad`.
__device__ __forceinline__ u64 vb_value_at(const u8* sb, int q, bool& bad) {
    int len = 1;
    while (len < 6 && (sb[q - len] & 0x80u)) len++;
    if (len > 5) {
        bad = true;
        len = 5;
    }
    // sb[q] holds the most significant group, sb[q - len + 1] the least
    u64 x = 0;
    for (int j = 0; j < len; j++) x = (x << 7) | (u64)(sb[q - j] & 0x7Fu);
    if (x >= (1ull << 32)) bad = true;
    return x;
}

// Decodes the nb-byte stream `in` into exactly n values with lo <= v < hi.
// Values: vals[0 .. n).  Rule lengths (kLens): offs[0 .. n] with offs[0] = 0
// and offs[r + 1] = offs[r] + length r; their sum must be `expect_sum`.
template <bool kLens>
__global__ void __launch_bounds__(kVbThreads) k_vb_decode(const u8* __restrict__ in, u64 nb, u64 n, u64 lo, u64 hi,
                                                          u64 expect_sum, u32* __restrict__ vals,
                                                          u64* __restrict__ offs, LBSlot<2>* lb, u64 epoch, u64* ctr,
                                                          u64 ctr_base, DevStatus* ds) {
    __shared__ __align__(16) u8 s_b[kVbHalo + kVbDecTile];
    __shared__ u64 s_v[kVbDecTile];
    pdl_wait();
    const u64 tile = dynamic_tile(ctr, ctr_base);
    const u64 t0 = tile * (u64)kVbDecTile;
    const u64 p0 = t0 + (u64)threadIdx.x * kVbBytes;
    // stage the tile (bytes past the stream read as 0) and the halo before it
    // (bytes before the stream read as 0: an end byte stops a backward walk)
    u8* sb = s_b + kVbHalo + threadIdx.x * kVbBytes;
    if (p0 + kVbBytes <= nb && (reinterpret_cast<uintptr_t>(in + p0) & 7) == 0) {
        const uint2 a = __ldg(reinterpret_cast<const uint2*>(in + p0));
        const uint2 b = __ldg(reinterpret_cast<const uint2*>(in + p0) + 1);
        reinterpret_cast<uint2*>(sb)[0] = a;
        reinterpret_cast<uint2*>(sb)[1] = b;
    } else {
#pragma unroll
        for (int q = 0; q < kVbBytes; q++) sb[q] = (p0 + q < nb) ? __ldg(in + p0 + q) : (u8)0;
    }
    if (threadIdx.x < kVbHalo) {
        const long long p = (long long)t0 - kVbHalo + (long long)threadIdx.x;
        s_b[threadIdx.x] = (p >= 0) ? __ldg(in + p) : (u8)0;
    }
    __syncthreads();
    // values ending in this thread's bytes: count (and, for lengths, sum)
    u32 ends = 0;
#pragma unroll
    for (int q = 0; q < kVbBytes; q++)
        if (p0 + q < nb && (sb[q] & 0x80u) == 0) ends |= 1u << q;
    const u32 cnt = __popc(ends);
    u64 sum = 0;
    bool bad = false;
    if (kLens) {
        for (u32 m = ends; m; m &= m - 1) {
            const u64 x = vb_value_at(sb, __ffs(m) - 1, bad);
            sum += x;
        }
    }
    // the stream must end with a value's last byte
    if (nb > 0 && p0 <= nb - 1 && nb - 1 < p0 + kVbBytes && (sb[nb - 1 - p0] & 0x80u)) bad = true;
    u64 tile_cnt, tile_sum = 0;
    const u64 my_cnt = block_excl_scan(cnt, tile_cnt);
    u64 my_sum = 0;
    if (kLens) my_sum = block_excl_scan(sum, tile_sum);
    u64 agg[2] = {tile_cnt, tile_sum}, excl[2];
    block_lookback<2>(lb, tile, epoch, agg, excl, ds);
    // stage values (or running offsets) in index order, then store coalesced
    {
        u64 run = my_sum;
        u32 i = (u32)my_cnt;
        for (u32 m = ends; m; m &= m - 1) {
            const u64 x = vb_value_at(sb, __ffs(m) - 1, bad);
            if (x < lo || x >= hi) bad = true;
            s_v[i++] = kLens ? run : x;
            run += x;
        }
    }
    if (bad) set_error(ds, kErrFormat);
    __syncthreads();
    for (u32 i = threadIdx.x; i < (u32)tile_cnt; i += kVbThreads) {
        const u64 idx = excl[0] + i;
        if (idx < n) {
            if (kLens) offs[idx] = excl[1] + s_v[i];
            else vals[idx] = (u32)s_v[i];
        }
    }
    if (t0 + kVbDecTile >= nb && threadIdx.x == 0) {
        const u64 total = excl[0] + tile_cnt;
        if (total != n) set_error(ds, kErrFormat);
        if (kLens) {
            const u64 s = excl[1] + tile_sum;
            if (s != expect_sum) set_error(ds, kErrFormat);
            if (total == n) offs[n] = s;
        }
    }
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------

static unsigned vb_grid(u64 n, u64 per) {
    u64 t = (n + per - 1) / per;
    return (unsigned)(t ? t : 1);
}

u64 vb_encode_tiles(u64 n) { return vb_grid(n, kVbTile); }
u64 vb_decode_tiles(u64 nb) { return vb_grid(nb, kVbDecTile); }

cudaError_t launch_vb_count(const u32* vals, const u64* offs, u64 n, u64* total, int sms, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<u64>((n + kVbThreads - 1) / kVbThreads, (u64)sms * 8);
    if (offs) return launch_pdl(k_vb_count<true>, grid, kVbThreads, st, vals, offs, n, total);
    return launch_pdl(k_vb_count<false>, grid, kVbThreads, st, vals, offs, n, total);
}

cudaError_t launch_vb_encode(const u32* vals, const u64* offs, u64 n, u8* out, u64* nbytes_out, bool pad, void* lb,
                             u64 epoch, u64* ctr, u64 ctr_base, DevStatus* ds, cudaStream_t st, u64* grid_out) {
    const unsigned grid = vb_grid(n, kVbTile);
    *grid_out = grid;
    if (offs)
        return launch_pdl(k_vb_encode<true>, grid, kVbThreads, st, vals, offs, n, out, nbytes_out, pad,
                          (LBSlot<2>*)lb, epoch, ctr, ctr_base, ds);
    return launch_pdl(k_vb_encode<false>, grid, kVbThreads, st, vals, offs, n, out, nbytes_out, pad, (LBSlot<2>*)lb,
                      epoch, ctr, ctr_base, ds);
}

cudaError_t launch_vb_decode(const u8* in, u64 nb, u64 n, u64 lo, u64 hi, u64 expect_sum, u32* vals, u64* offs,
                             void* lb, u64 epoch, u64* ctr, u64 ctr_base, DevStatus* ds, cudaStream_t st,
                             u64* grid_out) {
    const unsigned grid = vb_grid(nb, kVbDecTile);
    *grid_out = grid;
    if (offs)
        return launch_pdl(k_vb_decode<true>, grid, kVbThreads, st, in, nb, n, lo, hi, expect_sum, vals, offs,
                          (LBSlot<2>*)lb, epoch, ctr, ctr_base, ds);
    return launch_pdl(k_vb_decode<false>, grid, kVbThreads, st, in, nb, n, lo, hi, expect_sum, vals, offs,
                      (LBSlot<2>*)lb, epoch, ctr, ctr_base, ds);
}

}  // namespace lcg
