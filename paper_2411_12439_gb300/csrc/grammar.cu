// Kernels that work on finished grammars: MergeGrams (Sec. 3.6), the
// expansion exp(C[j]) (Sec. 2.2), and a generic two-column exclusive scan.
#include "lcg_dev.cuh"
#include "lcg_internal.h"
#include "table.cuh"

namespace lcg {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// --------------------------------------------------------------------------
// exclusive scan of two uint32 columns into uint64 (single pass)
// --------------------------------------------------------------------------

// kScanItems consecutive values of a column from p0 (16-byte loads when the
// whole run is inside the column and aligned), zero past n or for no column.
__device__ __forceinline__ void scan_load(const u32* in, u64 p0, u64 n, u32 (&v)[kScanItems]) {
    if (in != nullptr && p0 + kScanItems <= n && (reinterpret_cast<unsigned long long>(in + p0) & 15) == 0) {
#pragma unroll
        for (int q = 0; q < kScanItems / 4; q++) {
            const uint4 x = reinterpret_cast<const uint4*>(in + p0)[q];
            v[4 * q] = x.x, v[4 * q + 1] = x.y, v[4 * q + 2] = x.z, v[4 * q + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int it = 0; it < kScanItems; it++) v[it] = (in != nullptr && p0 + it < n) ? in[p0 + it] : 0u;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan2(const u32* __restrict__ in0, const u32* __restrict__ in1,
                                                        u64 n, u64* __restrict__ out0, u64* __restrict__ out1,
                                                        u64* __restrict__ totals, LBSlot<2>* lb, u64 epoch, u64* ctr,
                                                        u64 ctr_base, DevStatus* ds, const u64* n_dev) {
    pdl_wait();
    const u64 tile = dynamic_tile(ctr, ctr_base);
    if (n_dev != nullptr) n = min(*n_dev, n);
    if (tile > 0 && tile * (u64)kScanTile >= n) return;  // beyond the count read on the device
    const u64 p0 = tile * (u64)kScanTile + (u64)threadIdx.x * kScanItems;
    u32 a[kScanItems], b[kScanItems];
    scan_load(in0, p0, n, a);
    scan_load(in1, p0, n, b);
    u64 sa = 0, sb = 0;
#pragma unroll
    for (int it = 0; it < kScanItems; it++) {
        sa += a[it];
        sb += b[it];
    }
    u64 ta, tb;
    u64 ea = block_excl_scan(sa, ta);
    u64 eb = block_excl_scan(sb, tb);
    u64 agg[2] = {ta, tb}, excl[2];
    block_lookback<2>(lb, tile, epoch, agg, excl, ds);
    ea += excl[0];
    eb += excl[1];
#pragma unroll
    for (int it = 0; it < kScanItems; it++) {
        const u64 p = p0 + it;
        if (p < n) {
            out0[p] = ea;
            if (out1 != nullptr) out1[p] = eb;
        }
        ea += a[it];
        eb += b[it];
    }
    if ((tile + 1) * (u64)kScanTile >= n && threadIdx.x == 0) {
        totals[0] = excl[0] + ta;
        totals[1] = excl[1] + tb;
    }
}

u64 scan2_tiles_for(u64 n) { return (n + kScanTile - 1) / kScanTile; }
size_t scan2_lb_bytes(u64 tiles) { return scan2_lb_bytes_static(tiles); }

cudaError_t launch_scan2(const u32* in0, const u32* in1, u64 n, u64* out0, u64* out1, u64* totals, void* lb,
                         u64 epoch, u64* ctr, u64 ctr_base, DevStatus* ds, cudaStream_t st, u64* grid_out,
                         const u64* n_dev) {
    u64 tiles = scan2_tiles_for(n);
    if (tiles == 0) tiles = 1;
    *grid_out = tiles;
    return launch_pdl(k_scan2, (unsigned)tiles, kScanThreads, st, in0, in1, n, out0, out1, totals, (LBSlot<2>*)lb,
                      epoch, ctr, ctr_base, ds, n_dev);
}

// --------------------------------------------------------------------------
// MergeGrams
// --------------------------------------------------------------------------

// out[x] = M[in[x]]: rewrite right-hand sides of G_b into G_a's ranks.
__global__ void k_remap(const u32* __restrict__ in, u64 n, const u32* __restrict__ M, u32* __restrict__ out) {
    for (u64 x = blockIdx.x * (u64)blockDim.x + threadIdx.x; x < n; x += (u64)gridDim.x * blockDim.x)
        out[x] = M[in[x]];
}

// For every rule of G_b (right-hand side already over G_a's ranks): its rank
// in G_a when G_a has the same right-hand side (looked up in G_a's table of
// the level, hashed keys confirmed by comparing contents), else a miss.
template <bool kByte>
__global__ void k_merge_lookup(const u32* __restrict__ brhs, const u64* __restrict__ brhs_off,
                               const u32* __restrict__ bF, u64 gb, const u32* __restrict__ aFprev, LevelHash lh,
                               ContentTable at, const u32* __restrict__ arhs, const u64* __restrict__ arhs_off,
                               const u32* __restrict__ aF, u32* __restrict__ M, u32* __restrict__ miss,
                               u32* __restrict__ mlen, DevStatus* ds) {
    for (u64 r = blockIdx.x * (u64)blockDim.x + threadIdx.x; r < gb; r += (u64)gridDim.x * blockDim.x) {
        const u64 s = brhs_off[r], e = brhs_off[r + 1], len = e - s;
        u64 H = 0;
        for (u64 x = e; x-- > s;) H = addmod61(mulmod61(H, lh.c), (u64)__ldg(aFprev + brhs[x]));
        const int w = kByte ? 8 : kRankBits;
        const bool hashed = len > inline_max(w);
        const Key128 key = hashed ? key_hashed(H, len, 0) : key_inline([&](u64 j) { return brhs[s + j]; }, len, w);
        u64 found = ~0ull;
        if (at.cap) {
            found = table_find(at, key, hashed, [&](u64 ra) {
                const u64 o = arhs_off[ra];
                if (arhs_off[ra + 1] - o != len) return false;
                for (u64 x = 0; x < len; x++)
                    if (arhs[o + x] != brhs[s + x]) return false;
                return true;
            });
        }
        if (found != ~0ull) {
            if (aF[found] != bF[r]) set_error(ds, kErrMismatch);
            M[r] = (u32)found;
            miss[r] = 0;
            mlen[r] = 0;
        } else {
            miss[r] = 1;
            mlen[r] = (u32)len;
        }
    }
}

// Append the missed rules of G_b to G_a in G_b's rank order.
__global__ void k_merge_append(const u32* __restrict__ brhs, const u64* __restrict__ brhs_off,
                               const u32* __restrict__ bF, u64 gb, const u32* __restrict__ miss,
                               const u64* __restrict__ xrank, const u64* __restrict__ xlen, u64 ga, u64 Ga,
                               u32* __restrict__ arhs, u64* __restrict__ arhs_off, u32* __restrict__ aF,
                               u32* __restrict__ M) {
    for (u64 r = blockIdx.x * (u64)blockDim.x + threadIdx.x; r < gb; r += (u64)gridDim.x * blockDim.x) {
        if (!miss[r]) continue;
        const u64 nr = ga + xrank[r], o = Ga + xlen[r];
        const u64 s = brhs_off[r], e = brhs_off[r + 1];
        arhs_off[nr] = o;
        for (u64 x = s; x < e; x++) arhs[o + (x - s)] = brhs[x];
        aF[nr] = bF[r];
        M[r] = (u32)nr;
    }
}

__global__ void k_set_u64(u64* p, u64 v) { *p = v; }

// F^0[s] = h^0(s) = ((a_0 s + b_0) mod p) mod m for every byte s (Sec. 3.2).
__global__ void k_h0(LevelHash h0, u32* __restrict__ F0) {
    pdl_wait();
    const u32 s = threadIdx.x;
    if (s < 256) F0[s] = (u32)(addmod61(mulmod61(h0.a, (u64)s), h0.b) & h0.mmask);
}

cudaError_t launch_h0(LevelHash h0, u32* F0, cudaStream_t st) {
    return launch_pdl(k_h0, 1, 256, st, h0, F0);
}

// C_b entries of level `level` move to G_a's ranks.
// Imported rules: F^i[r] must be h^i of the rule's right-hand side
// (Eq. fast_hash over F^{i-1}); a difference means the grammar was built with
// another hash family (or was altered).
__global__ void k_check_fp(const u32* __restrict__ rhs, const u64* __restrict__ rhs_off, u64 g,
                           const u32* __restrict__ Fprev, LevelHash lh, const u32* __restrict__ F, DevStatus* ds) {
    for (u64 r = blockIdx.x * (u64)blockDim.x + threadIdx.x; r < g; r += (u64)gridDim.x * blockDim.x) {
        const u64 s = rhs_off[r], e = rhs_off[r + 1];
        u64 H = 0;
        for (u64 y = e; y-- > s;) H = addmod61(mulmod61(H, lh.c), (u64)__ldg(Fprev + rhs[y]));
        if (finish_hash(lh, H) != F[r]) set_error(ds, kErrMismatch);
    }
}

cudaError_t launch_check_fp(const u32* rhs, const u64* rhs_off, u64 g, const u32* Fprev, LevelHash lh, const u32* F,
                            DevStatus* ds, cudaStream_t st) {
    if (g == 0) return cudaSuccess;
    const u64 b = (g + 255) / 256;
    k_check_fp<<<(unsigned)(b < 152 * 16 ? b : 152 * 16), 256, 0, st>>>(rhs, rhs_off, g, Fprev, lh, F, ds);
    return cudaGetLastError();
}

// Root of strings j0 .. j0+cnt-1: C[j] = (level, rank) and the fingerprint
// F^level[rank] of exp(T_j) (Eq. fast_hash: it depends on the content only).
__global__ void k_roots(const u32* __restrict__ c_level, const u32* __restrict__ c_rank, u32 j0, u32 cnt, FTable ft,
                        u32* __restrict__ out) {
    for (u32 x = blockIdx.x * blockDim.x + threadIdx.x; x < cnt; x += gridDim.x * blockDim.x) {
        const u32 lvl = c_level[j0 + x], r = c_rank[j0 + x];
        out[3 * x] = lvl;
        out[3 * x + 1] = r;
        out[3 * x + 2] = lvl < ft.n ? __ldg(ft.F[lvl] + r) : 0u;
    }
}

cudaError_t launch_roots(const u32* c_level, const u32* c_rank, u32 j0, u32 cnt, const FTable& ft, u32* out,
                         cudaStream_t st) {
    if (cnt == 0) return cudaSuccess;
    k_roots<<<(cnt + 255) / 256 < 1024 ? (cnt + 255) / 256 : 1024, 256, 0, st>>>(c_level, c_rank, j0, cnt, ft, out);
    return cudaGetLastError();
}

__global__ void k_remap_c(const u32* __restrict__ c_level, u32* __restrict__ c_rank, u32 k, u32 level,
                          const u32* __restrict__ M) {
    for (u32 j = blockIdx.x * blockDim.x + threadIdx.x; j < k; j += gridDim.x * blockDim.x)
        if (c_level[j] == level) c_rank[j] = M[c_rank[j]];
}

static unsigned grid_for(u64 n, unsigned cap = 152 * 32) {
    u64 b = (n + 255) / 256;
    if (b == 0) b = 1;
    return (unsigned)(b < cap ? b : cap);
}

cudaError_t launch_remap(const u32* in, u64 n, const u32* M, u32* out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_remap<<<grid_for(n), 256, 0, st>>>(in, n, M, out);
    return cudaGetLastError();
}

cudaError_t launch_merge_lookup(const u32* brhs, const u64* brhs_off, const u32* bF, u64 gb, bool bytes,
                                const u32* aFprev, LevelHash lh, void* aslots, u64 acap, const u32* arhs,
                                const u64* arhs_off, const u32* aF, u32* M, u32* miss, u32* mlen, DevStatus* ds,
                                cudaStream_t st) {
    if (gb == 0) return cudaSuccess;
    const ContentTable at{(Slot*)aslots, acap};
    if (bytes)
        k_merge_lookup<true><<<grid_for(gb), 256, 0, st>>>(brhs, brhs_off, bF, gb, aFprev, lh, at, arhs, arhs_off, aF,
                                                           M, miss, mlen, ds);
    else
        k_merge_lookup<false><<<grid_for(gb), 256, 0, st>>>(brhs, brhs_off, bF, gb, aFprev, lh, at, arhs, arhs_off,
                                                            aF, M, miss, mlen, ds);
    return cudaGetLastError();
}

cudaError_t launch_merge_append(const u32* brhs, const u64* brhs_off, const u32* bF, u64 gb, const u32* miss,
                                const u64* xrank, const u64* xlen, u64 ga, u64 Ga, u32* arhs, u64* arhs_off,
                                u32* aF, u32* M, u64 ga_new, u64 Ga_new, cudaStream_t st) {
    if (gb > 0)
        k_merge_append<<<grid_for(gb), 256, 0, st>>>(brhs, brhs_off, bF, gb, miss, xrank, xlen, ga, Ga, arhs,
                                                     arhs_off, aF, M);
    k_set_u64<<<1, 1, 0, st>>>(arhs_off + ga_new, Ga_new);
    return cudaGetLastError();
}

cudaError_t launch_remap_c(const u32* c_level, u32* c_rank, u32 k, u32 level, const u32* M, cudaStream_t st) {
    if (k == 0) return cudaSuccess;
    k_remap_c<<<grid_for(k, 152), 256, 0, st>>>(c_level, c_rank, k, level, M);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// exp(C[j]): top-down expansion, one level per step
// --------------------------------------------------------------------------

__global__ void k_rule_lens(const u32* __restrict__ cur, u64 cnt, const u64* __restrict__ rhs_off,
                            u32* __restrict__ lens) {
    for (u64 x = blockIdx.x * (u64)blockDim.x + threadIdx.x; x < cnt; x += (u64)gridDim.x * blockDim.x) {
        const u32 r = cur[x];
        lens[x] = (u32)(rhs_off[r + 1] - rhs_off[r]);
    }
}

__global__ void k_expand(const u32* __restrict__ cur, u64 cnt, const u64* __restrict__ offs,
                         const u64* __restrict__ rhs_off, const u32* __restrict__ rhs, u32* __restrict__ next) {
    for (u64 x = blockIdx.x * (u64)blockDim.x + threadIdx.x; x < cnt; x += (u64)gridDim.x * blockDim.x) {
        const u32 r = cur[x];
        const u64 s = rhs_off[r], e = rhs_off[r + 1], o = offs[x];
        for (u64 y = s; y < e; y++) next[o + (y - s)] = rhs[y];
    }
}

__global__ void k_to_bytes(const u32* __restrict__ cur, u64 cnt, unsigned char* __restrict__ out) {
    for (u64 x = blockIdx.x * (u64)blockDim.x + threadIdx.x; x < cnt; x += (u64)gridDim.x * blockDim.x)
        out[x] = (unsigned char)cur[x];
}

cudaError_t launch_rule_lens(const u32* cur, u64 cnt, const u64* rhs_off, u32* lens, cudaStream_t st) {
    k_rule_lens<<<grid_for(cnt), 256, 0, st>>>(cur, cnt, rhs_off, lens);
    return cudaGetLastError();
}

cudaError_t launch_expand(const u32* cur, u64 cnt, const u64* offs, const u64* rhs_off, const u32* rhs, u32* next,
                          cudaStream_t st) {
    k_expand<<<grid_for(cnt), 256, 0, st>>>(cur, cnt, offs, rhs_off, rhs, next);
    return cudaGetLastError();
}

cudaError_t launch_to_bytes(const u32* cur, u64 cnt, unsigned char* out, cudaStream_t st) {
    k_to_bytes<<<grid_for(cnt), 256, 0, st>>>(cur, cnt, out);
    return cudaGetLastError();
}

}  // namespace lcg
