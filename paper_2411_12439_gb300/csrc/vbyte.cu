// VByte codec of the grammar's arrays (Sec. 4, resource usage: rules stored
// with VBytes instead of 32-bit cells).  A value is cut into groups of 7 bits,
// least significant group first, one group per byte; the high bit of a byte
// is set when another byte of the same value follows (the LEB128 / varint
// layout).
//
// Both directions run in three independent streaming steps, with no wait of
// one tile on another:
//   encode: k_vb_tile_bytes (stream bytes of each tile of 2048 values), an
//     exclusive scan of those counts (k_scan2), k_vb_write (each tile
//     re-reads its values, assembles its bytes in shared memory and stores
//     them at its offset with 4-byte stores, the edges byte by byte).  An
//     export needs the counts anyway to lay out its sections.
//   decode: k_vb_tile_ends (values ending in each tile of 4096 stream bytes),
//     a scan of those counts, k_vb_dwrite (every byte without the high bit
//     ends a value, which is assembled in registers from the bytes before it;
//     the tile's values are staged and stored coalesced at its offset).  Malformed streams (a value of more
//     than 32 bits or 5 bytes, a stream that ends inside a value, a value
//     outside the allowed range, another number of values) set kErrFormat;
//     no write leaves the output.
// k_vb_count sizes a column without writing it (lcg_vbyte_size).
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
// encode: bytes per tile, (scan of the tile counts), write
// --------------------------------------------------------------------------

// Values of this thread (kVbItems from p0; 0 past n).
template <bool kLens>
__device__ __forceinline__ void vb_load(const u32* vals, const u64* offs, u64 n, u64 p0, u32 (&v)[kVbItems]) {
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
}

template <bool kLens>
__device__ __forceinline__ u32 vb_thread_bytes(const u32 (&v)[kVbItems], u64 n, u64 p0) {
    u32 b = 0;
#pragma unroll
    for (int it = 0; it < kVbItems; it++) b += (p0 + it < n) ? vb_len(v[it]) : 0u;
    return b;
}

// tile_bytes[t] = bytes of the VByte stream of values [t * kVbTile, ...).
template <bool kLens>
__global__ void __launch_bounds__(kVbThreads) k_vb_tile_bytes(const u32* __restrict__ vals,
                                                              const u64* __restrict__ offs, u64 n,
                                                              u32* __restrict__ tile_bytes) {
    pdl_wait();
    const u64 p0 = blockIdx.x * (u64)kVbTile + (u64)threadIdx.x * kVbItems;
    u32 v[kVbItems];
    vb_load<kLens>(vals, offs, n, p0, v);
    u32 b = vb_thread_bytes<kLens>(v, n, p0);
    for (int o = 16; o > 0; o >>= 1) b += __shfl_down_sync(0xffffffffu, b, o);
    __shared__ u32 s_w[kVbThreads / 32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        u32 t = 0;
        for (int w = 0; w < kVbThreads / 32; w++) t += s_w[w];
        tile_bytes[blockIdx.x] = t;
    }
}

// Store a tile's tb stream bytes (assembled in s_out) at dst: the bytes up to
// a 4-byte boundary and after the last whole word one by one, the rest as
// 4-byte words.
__device__ __forceinline__ void vb_store_tile(u8* dst, const u8* s_out, u32 tb) {
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
}

// Writes the VByte stream of the n values to out[0 ..): tile t at its
// offset tile_off[t] (exclusive scan of k_vb_tile_bytes), assembled in shared
// memory and stored with 4-byte stores (edges byte by byte).  With `pad`, the
// last tile adds zeros up to the next multiple of 8 bytes (section padding).
template <bool kLens>
__global__ void __launch_bounds__(kVbThreads) k_vb_write(const u32* __restrict__ vals, const u64* __restrict__ offs,
                                                         u64 n, const u64* __restrict__ tile_off,
                                                         u8* __restrict__ out, bool pad) {
    __shared__ u8 s_out[kVbTile * 5];
    pdl_wait();
    const u64 tile = blockIdx.x;
    const u64 p0 = tile * (u64)kVbTile + (u64)threadIdx.x * kVbItems;
    const u64 base = tile_off[tile];  // issued with the value loads, used after the assembly
    u32 v[kVbItems];
    vb_load<kLens>(vals, offs, n, p0, v);
    u64 tile_bytes;
    const u64 my_off = block_excl_scan(vb_thread_bytes<kLens>(v, n, p0), tile_bytes);
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
    vb_store_tile(out + base, s_out, (u32)tile_bytes);
    if (pad && tile == gridDim.x - 1 && threadIdx.x == 0)
        for (u64 z = base + tile_bytes; z & 7; z++) out[z] = 0;
}

// --------------------------------------------------------------------------
// decode: values per tile, (scan of the tile counts), write
// --------------------------------------------------------------------------

// High bit of each byte of a little-endian word: bit q = bit 7 of byte q
// (the eight bits gathered into the top byte by one multiplication).
__device__ __forceinline__ u32 vb_high_bits(u64 w) {
    return (u32)((((w & 0x8080808080808080ull) >> 7) * 0x0102040810204080ull) >> 56);
}

// Bytes [p0, p0 + 16) of the stream as two little-endian words (0 past nb),
// and the mask of those that end a value (bit q: byte p0 + q).
__device__ __forceinline__ u32 vb_load16(const u8* in, u64 nb, u64 p0, u64& w1, u64& w2) {
    if (p0 + kVbBytes <= nb && (reinterpret_cast<uintptr_t>(in + p0) & 7) == 0) {
        w1 = __ldg(reinterpret_cast<const unsigned long long*>(in + p0));
        w2 = __ldg(reinterpret_cast<const unsigned long long*>(in + p0) + 1);
    } else {
        w1 = w2 = 0;
#pragma unroll
        for (int q = 0; q < kVbBytes; q++) {
            const u64 x = (p0 + q < nb) ? (u64)__ldg(in + p0 + q) : 0ull;
            if (q < 8) w1 |= x << (8 * q);
            else w2 |= x << (8 * (q - 8));
        }
    }
    // a byte ends a value when its high bit is clear (bytes past nb do not)
    u32 m = ~(vb_high_bits(w1) | (vb_high_bits(w2) << 8)) & 0xFFFFu;
    if (p0 + kVbBytes > nb) m &= (p0 >= nb) ? 0u : ((1u << (u32)(nb - p0)) - 1u);
    return m;
}

// tile_cnt[t] = values that end in bytes [t * kVbDecTile, ...) of the stream.
__global__ void __launch_bounds__(kVbThreads) k_vb_tile_ends(const u8* __restrict__ in, u64 nb,
                                                             u32* __restrict__ tile_cnt) {
    pdl_wait();
    const u64 p0 = blockIdx.x * (u64)kVbDecTile + (u64)threadIdx.x * kVbBytes;
    u64 w1, w2;
    u32 c = __popc(vb_load16(in, nb, p0, w1, w2));
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    __shared__ u32 s_w[kVbThreads / 32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        u32 t = 0;
        for (int w = 0; w < kVbThreads / 32; w++) t += s_w[w];
        tile_cnt[blockIdx.x] = t;
    }
}

// Decodes the nb-byte stream into exactly n values with lo <= v < hi: the
// values ending in tile t go to vals[cnt_off[t] ...) (cnt_off: exclusive
// scan of k_vb_tile_ends).  Each thread holds its 16 bytes and the 8 before
// them (from the lane before, or the warp before, or global memory at a
// tile's start; zeros before the stream, which end no value's run) in three
// registers.  A value ending at window byte e takes the bytes after the last
// earlier end byte: its length is one more than the run of continuation bits
// right below e, and its groups come from the 8 bytes at e - 4 by one funnel
// shift.  The tile's values are staged in shared memory and stored coalesced.
// One tile of a stream (bytes [t0, t0 + 4096) of src, nb bytes in all) into
// out[base ...): each thread holds its 16 bytes and the 8 before them (from
// the lane before, the warp before, or global memory at the tile's start;
// zeros before the stream, which end no value's run) in three registers.  A
// value ending at window byte e takes the bytes after the last earlier end
// byte: its length is one more than the run of continuation bits right below
// e, and its groups come from the 8 bytes at e - 4 by one funnel shift.  The
// tile's values are staged in shared memory and stored coalesced.  `last`:
// the stream's last tile, which checks that n values were found.
__device__ __forceinline__ void vb_decode_tile(const u8* __restrict__ src, u64 nb, u64 n, u64 lo, u64 hi, u64 t0,
                                               u64 base, bool last, u32* __restrict__ out, u32* s_v, u64* s_tail,
                                               DevStatus* ds) {
    const u64 p0 = t0 + (u64)threadIdx.x * kVbBytes;
    const u32 lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // loads issued together: the 8 bytes before the tile (thread 0), the
    // thread's 16 bytes
    u64 before = 0;
    if (threadIdx.x == 0 && t0 > 0) {
        if ((reinterpret_cast<uintptr_t>(src + t0 - 8) & 7) == 0) {
            before = __ldg(reinterpret_cast<const unsigned long long*>(src + t0 - 8));
        } else {
#pragma unroll
            for (int q = 0; q < 8; q++) before |= (u64)__ldg(src + t0 - 8 + q) << (8 * q);
        }
    }
    u64 w1, w2;
    const u32 ends = vb_load16(src, nb, p0, w1, w2);
    u64 w0 = __shfl_up_sync(0xffffffffu, w2, 1);  // the 8 bytes before p0
    if (lane == 31) s_tail[wid] = w2;
    u64 tile_cnt;
    const u64 my_cnt = block_excl_scan(__popc(ends), tile_cnt);  // its barriers also publish s_tail
    if (lane == 0) w0 = (wid > 0) ? s_tail[wid - 1] : before;
    // continuation bits of the 24-byte window (bit j: window byte j)
    const u32 cont = vb_high_bits(w0) | (vb_high_bits(w1) << 8) | (vb_high_bits(w2) << 16);
    bool bad = false;
    // the stream must end with a value's last byte
    if (p0 <= nb - 1 && nb - 1 < p0 + kVbBytes && !((ends >> (u32)(nb - 1 - p0)) & 1u)) bad = true;
    u32 i = (u32)my_cnt;
    for (u32 m = ends; m; m &= m - 1) {
        const u32 e = (u32)__ffs(m) - 1 + 8;           // window byte of the value's last byte, 8 .. 23
        const u32 run = __clz(~(cont << (32 - e)));     // continuation bytes right before it
        u32 len = run + 1;
        if (len > 5) {
            bad = true;
            len = 5;
        }
        // the 8 window bytes from e - 4 (4 .. 19): one funnel shift of two words
        const u32 st = e - 4, sh = (st & 7) * 8;
        const u64 lo_w = (st < 8) ? w0 : (st < 16 ? w1 : w2);
        const u64 hi_w = (st < 8) ? w1 : (st < 16 ? w2 : 0ull);
        const u64 v8 = sh ? ((lo_w >> sh) | (hi_w << (64 - sh))) : lo_w;
        // five 7-bit groups, the least significant from byte e - 4
        const u64 y = (v8 & 0x7Full) | ((v8 >> 1) & 0x3F80ull) | ((v8 >> 2) & 0x1FC000ull) |
                      ((v8 >> 3) & 0xFE00000ull) | ((v8 >> 4) & 0x7F0000000ull);
        const u64 x = y >> (7 * (5 - len));
        if (x >= (1ull << 32) || x < lo || x >= hi) bad = true;
        s_v[i++] = (u32)x;
    }
    if (bad) set_error(ds, kErrFormat);
    __syncthreads();
    for (u32 k = threadIdx.x; k < (u32)tile_cnt; k += kVbThreads) {
        const u64 idx = base + k;
        if (idx < n) out[idx] = s_v[k];
    }
    if (last && threadIdx.x == 0 && base + tile_cnt != n) set_error(ds, kErrFormat);
}

// Decodes the nb-byte stream into exactly n values with lo <= v < hi: the
// values ending in tile t go to vals[cnt_off[t] ...) (cnt_off: exclusive
// scan of k_vb_tile_ends).
__global__ void __launch_bounds__(kVbThreads) k_vb_dwrite(const u8* __restrict__ in, u64 nb, u64 n, u64 lo, u64 hi,
                                                          const u64* __restrict__ cnt_off, u32* __restrict__ vals,
                                                          DevStatus* ds) {
    __shared__ u32 s_v[kVbDecTile];
    __shared__ u64 s_tail[kVbThreads / 32];
    pdl_wait();
    const u64 tile = blockIdx.x;
    vb_decode_tile(in, nb, n, lo, hi, tile * (u64)kVbDecTile, cnt_off[tile], tile == gridDim.x - 1, vals, s_v,
                   s_tail, ds);
}

// --------------------------------------------------------------------------
// every column of a grammar in one launch per step
// --------------------------------------------------------------------------
//
// Tile t of a launch belongs to column c with cols[c].tile0 <= t <
// cols[c + 1].tile0 (the last entry is a sentinel holding the launch's tile
// count); a block finds its column by binary search over the tile0 values,
// loaded into shared memory.

template <typename Col>
__device__ __forceinline__ u32 vb_column_of(const Col* cols, u32 ncols, u64 t, u64* s_t0) {
    for (u32 c = threadIdx.x; c <= ncols; c += blockDim.x) s_t0[c] = cols[c].tile0;
    __syncthreads();
    u32 lo = 0, hi = ncols;  // s_t0[lo] <= t < s_t0[hi]
    while (hi - lo > 1) {
        const u32 mid = (lo + hi) / 2;
        if (s_t0[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kVbThreads) k_vb_tile_bytes_all(const VbEncCol* __restrict__ cols, u32 ncols,
                                                                  u32* __restrict__ tile_bytes,
                                                                  u64* __restrict__ col_bytes) {
    __shared__ u64 s_t0[kVbMaxCols + 1];
    __shared__ u32 s_w[kVbThreads / 32];
    pdl_wait();
    const u64 t = blockIdx.x;
    const u32 c = vb_column_of(cols, ncols, t, s_t0);
    const VbEncCol col = cols[c];
    const u64 p0 = (t - col.tile0) * (u64)kVbTile + (u64)threadIdx.x * kVbItems;
    u32 v[kVbItems];
    u32 b;
    if (col.offs) {
        vb_load<true>(col.vals, col.offs, col.n, p0, v);
        b = vb_thread_bytes<true>(v, col.n, p0);
    } else {
        vb_load<false>(col.vals, col.offs, col.n, p0, v);
        b = vb_thread_bytes<false>(v, col.n, p0);
    }
    for (int o = 16; o > 0; o >>= 1) b += __shfl_down_sync(0xffffffffu, b, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        u32 sum = 0;
        for (int w = 0; w < kVbThreads / 32; w++) sum += s_w[w];
        tile_bytes[t] = sum;
        if (sum) atomicAdd(reinterpret_cast<unsigned long long*>(col_bytes + c), (unsigned long long)sum);
    }
}

// Tile t of column c goes to cols[c].dst + tile_off[t] - tile_off[cols[c].tile0];
// the last tile of each column zero-pads it to a multiple of 8 bytes.
__global__ void __launch_bounds__(kVbThreads) k_vb_write_all(const VbEncCol* __restrict__ cols, u32 ncols,
                                                             const u64* __restrict__ tile_off) {
    __shared__ u64 s_t0[kVbMaxCols + 1];
    __shared__ u8 s_out[kVbTile * 5];
    pdl_wait();
    const u64 t = blockIdx.x;
    const u32 c = vb_column_of(cols, ncols, t, s_t0);
    const VbEncCol col = cols[c];
    const u64 base = tile_off[t] - tile_off[col.tile0];
    const bool last = (t + 1 == s_t0[c + 1]);
    const u64 p0 = (t - col.tile0) * (u64)kVbTile + (u64)threadIdx.x * kVbItems;
    u32 v[kVbItems];
    u32 mine;
    if (col.offs) {
        vb_load<true>(col.vals, col.offs, col.n, p0, v);
        mine = vb_thread_bytes<true>(v, col.n, p0);
    } else {
        vb_load<false>(col.vals, col.offs, col.n, p0, v);
        mine = vb_thread_bytes<false>(v, col.n, p0);
    }
    u64 tile_bytes;
    const u64 my_off = block_excl_scan(mine, tile_bytes);
    u32 o = (u32)my_off;
#pragma unroll
    for (int it = 0; it < kVbItems; it++) {
        if (p0 + it < col.n) {
            u32 x = v[it];
            while (x >= 0x80u) {
                s_out[o++] = (u8)(x | 0x80u);
                x >>= 7;
            }
            s_out[o++] = (u8)x;
        }
    }
    __syncthreads();
    vb_store_tile(col.dst + base, s_out, (u32)tile_bytes);
    if (last && threadIdx.x == 0)
        for (u64 z = base + tile_bytes; z & 7; z++) col.dst[z] = 0;
}

__global__ void __launch_bounds__(kVbThreads) k_vb_tile_ends_all(const VbDecCol* __restrict__ cols, u32 ncols,
                                                                 u32* __restrict__ tile_cnt) {
    __shared__ u64 s_t0[kVbMaxCols + 1];
    __shared__ u32 s_w[kVbThreads / 32];
    pdl_wait();
    const u64 t = blockIdx.x;
    const u32 c = vb_column_of(cols, ncols, t, s_t0);
    const VbDecCol col = cols[c];
    const u64 p0 = (t - col.tile0) * (u64)kVbDecTile + (u64)threadIdx.x * kVbBytes;
    u64 w1, w2;
    u32 n = __popc(vb_load16(col.src, col.nb, p0, w1, w2));
    for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        u32 sum = 0;
        for (int w = 0; w < kVbThreads / 32; w++) sum += s_w[w];
        tile_cnt[t] = sum;
    }
}

__global__ void __launch_bounds__(kVbThreads) k_vb_dwrite_all(const VbDecCol* __restrict__ cols, u32 ncols,
                                                              const u64* __restrict__ cnt_off, DevStatus* ds) {
    __shared__ u64 s_t0[kVbMaxCols + 1];
    __shared__ u32 s_v[kVbDecTile];
    __shared__ u64 s_tail[kVbThreads / 32];
    pdl_wait();
    const u64 t = blockIdx.x;
    const u32 c = vb_column_of(cols, ncols, t, s_t0);
    const VbDecCol col = cols[c];
    const bool last = (t + 1 == s_t0[c + 1]);
    const u64 base = cnt_off[t] - cnt_off[col.tile0];
    const u64 t0 = (t - col.tile0) * (u64)kVbDecTile;
    vb_decode_tile(col.src, col.nb, col.n, col.lo, col.hi, t0, base, last, col.out, s_v, s_tail, ds);
}

// Offsets of every level from the scan of all levels' rule lengths (levels
// with rules only, in order): rhs_off[r] = scan[gbase + r] - scan[gbase],
// rhs_off[g] = the level's length sum, which must be G (else kErrFormat).
// blockIdx.y = level; *total = the sum of all lengths.
__global__ void k_vb_offsets_all(const VbLevelOff* __restrict__ lv, const u64* __restrict__ scan,
                                 const u64* __restrict__ total, u32 nlv, DevStatus* ds) {
    pdl_wait();
    const VbLevelOff L = lv[blockIdx.y];
    const u64 s0 = scan[L.gbase];
    const u64 s1 = (blockIdx.y + 1 < nlv) ? scan[lv[blockIdx.y + 1].gbase] : *total;
    for (u64 r = blockIdx.x * (u64)blockDim.x + threadIdx.x; r <= L.g; r += (u64)gridDim.x * blockDim.x)
        L.rhs_off[r] = (r < L.g ? scan[L.gbase + r] : s1) - s0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && s1 - s0 != L.G) set_error(ds, kErrFormat);
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------

static u64 vb_tiles(u64 n, u64 per) { return (n + per - 1) / per; }

u64 vb_encode_tiles(u64 n) { return vb_tiles(n, kVbTile); }
u64 vb_decode_tiles(u64 nb) { return vb_tiles(nb, kVbDecTile); }

cudaError_t launch_vb_count(const u32* vals, const u64* offs, u64 n, u64* total, int sms, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<u64>((n + kVbThreads - 1) / kVbThreads, (u64)sms * 8);
    if (offs) return launch_pdl(k_vb_count<true>, grid, kVbThreads, st, vals, offs, n, total);
    return launch_pdl(k_vb_count<false>, grid, kVbThreads, st, vals, offs, n, total);
}

cudaError_t launch_vb_tile_bytes(const u32* vals, const u64* offs, u64 n, u32* tile_bytes, cudaStream_t st) {
    const unsigned grid = (unsigned)vb_encode_tiles(n);
    if (grid == 0) return cudaSuccess;
    if (offs) return launch_pdl(k_vb_tile_bytes<true>, grid, kVbThreads, st, vals, offs, n, tile_bytes);
    return launch_pdl(k_vb_tile_bytes<false>, grid, kVbThreads, st, vals, offs, n, tile_bytes);
}

cudaError_t launch_vb_write(const u32* vals, const u64* offs, u64 n, const u64* tile_off, u8* out, bool pad,
                            cudaStream_t st) {
    const unsigned grid = (unsigned)vb_encode_tiles(n);
    if (grid == 0) return cudaSuccess;
    if (offs) return launch_pdl(k_vb_write<true>, grid, kVbThreads, st, vals, offs, n, tile_off, out, pad);
    return launch_pdl(k_vb_write<false>, grid, kVbThreads, st, vals, offs, n, tile_off, out, pad);
}

cudaError_t launch_vb_tile_ends(const u8* in, u64 nb, u32* tile_cnt, cudaStream_t st) {
    const unsigned grid = (unsigned)vb_decode_tiles(nb);
    if (grid == 0) return cudaSuccess;
    return launch_pdl(k_vb_tile_ends, grid, kVbThreads, st, in, nb, tile_cnt);
}

cudaError_t launch_vb_dwrite(const u8* in, u64 nb, u64 n, u64 lo, u64 hi, const u64* cnt_off, u32* vals,
                             DevStatus* ds, cudaStream_t st) {
    const unsigned grid = (unsigned)vb_decode_tiles(nb);
    if (grid == 0) return cudaSuccess;
    return launch_pdl(k_vb_dwrite, grid, kVbThreads, st, in, nb, n, lo, hi, cnt_off, vals, ds);
}

cudaError_t launch_vb_tile_bytes_all(const VbEncCol* cols, u32 ncols, u64 tiles, u32* tile_bytes, u64* col_bytes,
                                     cudaStream_t st) {
    if (tiles == 0) return cudaSuccess;
    return launch_pdl(k_vb_tile_bytes_all, (unsigned)tiles, kVbThreads, st, cols, ncols, tile_bytes, col_bytes);
}

cudaError_t launch_vb_write_all(const VbEncCol* cols, u32 ncols, u64 tiles, const u64* tile_off, cudaStream_t st) {
    if (tiles == 0) return cudaSuccess;
    return launch_pdl(k_vb_write_all, (unsigned)tiles, kVbThreads, st, cols, ncols, tile_off);
}

cudaError_t launch_vb_tile_ends_all(const VbDecCol* cols, u32 ncols, u64 tiles, u32* tile_cnt, cudaStream_t st) {
    if (tiles == 0) return cudaSuccess;
    return launch_pdl(k_vb_tile_ends_all, (unsigned)tiles, kVbThreads, st, cols, ncols, tile_cnt);
}

cudaError_t launch_vb_dwrite_all(const VbDecCol* cols, u32 ncols, u64 tiles, const u64* cnt_off, DevStatus* ds,
                                 cudaStream_t st) {
    if (tiles == 0) return cudaSuccess;
    return launch_pdl(k_vb_dwrite_all, (unsigned)tiles, kVbThreads, st, cols, ncols, cnt_off, ds);
}

cudaError_t launch_vb_offsets_all(const VbLevelOff* lv, u32 nlv, u64 max_g, const u64* scan, const u64* total,
                                  DevStatus* ds, cudaStream_t st) {
    if (nlv == 0) return cudaSuccess;
    const unsigned gx = (unsigned)std::min<u64>((max_g + 1 + kVbThreads - 1) / kVbThreads, 4096);
    return launch_pdl(k_vb_offsets_all, dim3(gx, nlv), dim3(kVbThreads), st, lv, scan, total, nlv, ds);
}

}  // namespace lcg
