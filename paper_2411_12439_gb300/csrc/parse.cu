// Kernels of one BuildGram round (Sec. 3.3) over all active strings of a
// batch, and their host-side launchers.
//
// A round i reads the sequence T^i (bytes in round 1, uint32 ranks later) of
// the active strings, laid out back to back with offsets soff[0..k], and the
// fingerprints F^{i-1} of its symbols.  It runs:
//   k_breaks   symbol fingerprints + RandLMSPar break bits (Eq. rand_types),
//              one bit per position, and the phrase count of every tile
//              (decoupled look-back prefix sums)
//   k_strings  per-string phrase ranges; strings that become one phrase retire
//   k_phrases  per phrase: polynomial fingerprint h^i (Eq. fast_hash) and
//              insertion into the phrase table with content comparison
//   k_name     first-occurrence flags -> ranks (single-pass scan); writes the
//              level-i rules (rhs, rhs_off) and F^i
//   k_rewrite  T^{i+1}[p] = rank of phrase p, compacting retired strings
#include "lcg_dev.cuh"
#include "lcg_internal.h"

namespace lcg {

constexpr int kTilePos = 8192;            // positions per break/phrase tile
constexpr int kTileWords = kTilePos / 32; // one bitmap word per thread
constexpr int kNameThreads = 256;
constexpr int kNameItems = 4;
constexpr int kNameTile = kNameThreads * kNameItems;
constexpr u64 kNone = 1ull << 32;          // "no different fingerprint to the right"
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

// index of the string holding position `pos`: largest j with soff[j] <= pos
__device__ __forceinline__ u32 string_of(const u64* soff, u32 k, u64 pos) {
    u32 lo = 0, hi = k;  // answer in [lo, hi)
    while (hi - lo > 1) {
        u32 mid = (lo + hi) >> 1;
        if (__ldg(soff + mid) <= pos) lo = mid; else hi = mid;
    }
    return lo;
}

// --------------------------------------------------------------------------
// k_breaks
// --------------------------------------------------------------------------

template <typename T>
__device__ u64 scan_right_diff(const T* S, FpSource<T> fp, u64 from, u64 strend, u32 val) {
    for (u64 y = from; y < strend; y++) {
        u32 fy = fp(S[y]);
        if (fy != val) return fy;
    }
    return kNone;
}

template <typename T>
__global__ void __launch_bounds__(kTileWords) k_breaks(const T* __restrict__ S, u64 n, const u64* __restrict__ soff,
                                                       u32 k, const u32* __restrict__ Fprev,
                                                       u32* __restrict__ bitmap, u64* __restrict__ tile_base,
                                                       LBSlot<1>* lb, u64 epoch, u64* ctr, u64 ctr_base,
                                                       u64* total_out, DevStatus* ds) {
    __shared__ u32 sF[256];
    FpSource<T> fp;
    if constexpr (sizeof(T) == 1) {
        for (int x = threadIdx.x; x < 256; x += blockDim.x) sF[x] = Fprev[x];
        __syncthreads();
        fp.F = sF;
    } else {
        fp.F = Fprev;
    }
    const u64 tile = dynamic_tile(ctr, ctr_base);
    const u64 w = tile * kTileWords + threadIdx.x;
    const u64 base = w * 32;
    u32 word = 0;
    if (base < n) {
        const int cnt = (int)min((u64)32, n - base);
        u32 v[32];
#pragma unroll
        for (int b = 0; b < 32; b++) v[b] = (b < cnt) ? fp(S[base + b]) : 0u;
        const u32 prev = base > 0 ? fp(S[base - 1]) : 0u;
        const u64 nextpos = base + cnt;  // first position after this word
        const u32 nextv = nextpos < n ? fp(S[nextpos]) : 0u;
        // string starts among positions base .. base+32
        u32 j = string_of(soff, k, base);
        unsigned long long starts = 0;  // bit b: base + b starts a string (b <= 32)
        {
            u32 jj = j;
            if (__ldg(soff + jj) == base) starts |= 1ull;
            while (jj + 1 <= k) {
                u64 s = __ldg(soff + jj + 1);
                if (s > base + 32 || s >= n) break;
                starts |= 1ull << (s - base);
                jj++;
            }
        }
        // right to left: nd = first fingerprint right of b that differs from v[b]
        u64 nd;
        bool unknown = false;
        const int last = cnt - 1;
        if (nextpos >= n || ((starts >> (last + 1)) & 1)) nd = kNone;
        else if (nextv != v[last]) nd = nextv;
        else { nd = kNone; unknown = true; }
        for (int b = last; b >= 0; b--) {
            bool brk;
            if ((starts >> b) & 1) {
                brk = true;
            } else {
                const u32 left = b > 0 ? v[b - 1] : prev;
                brk = false;
                if (left > v[b]) {
                    if (unknown) {
                        // the run holding b reaches past this word: follow it
                        u32 jl = string_of(soff, k, base + last);
                        nd = scan_right_diff<T>(S, fp, nextpos, __ldg(soff + jl + 1), v[b]);
                        unknown = false;
                    }
                    brk = (nd != kNone) && (nd > (u64)v[b]);
                }
            }
            if (brk) word |= 1u << b;
            if (b > 0) {
                if ((starts >> b) & 1) { nd = kNone; unknown = false; }
                else if (v[b] != v[b - 1]) { nd = v[b]; unknown = false; }
            }
        }
        bitmap[w] = word;
    }
    u64 total;
    (void)block_excl_scan((u64)__popc(word), total);
    u64 agg[1] = {total}, excl[1];
    block_lookback<1>(lb, tile, epoch, agg, excl, ds);
    if (threadIdx.x == 0) {
        tile_base[tile] = excl[0];
        if ((tile + 1) * (u64)kTilePos >= n) *total_out = excl[0] + total;
    }
}

// --------------------------------------------------------------------------
// k_strings: per-string phrase ranges, retirement, next offsets (one block)
// --------------------------------------------------------------------------

__device__ u64 phrase_index_at(const u32* bitmap, const u64* tile_base, u64 pos) {
    u64 tile = pos / kTilePos;
    u64 w0 = tile * kTileWords, w = pos / 32;
    u64 idx = tile_base[tile];
    for (u64 x = w0; x < w; x++) idx += __popc(bitmap[x]);
    u32 bit = (u32)(pos & 31);
    idx += __popc(bitmap[w] & ((1u << bit) - 1u));
    return idx;
}

__global__ void __launch_bounds__(1024) k_strings(const u64* __restrict__ soff, const u32* __restrict__ sid, u32 k,
                                                  const u32* __restrict__ bitmap, const u64* __restrict__ tile_base,
                                                  const u64* __restrict__ total, u64* __restrict__ soff_next,
                                                  u32* __restrict__ sid_next, u64* __restrict__ R_phr,
                                                  u32* __restrict__ R_sid, RoundCounts* __restrict__ rc) {
    const u64 P = *total;
    u64 carry = 0;
    for (u32 j0 = 0; j0 < k; j0 += blockDim.x) {
        u32 j = j0 + threadIdx.x;
        u64 first = 0, nextf = 0;
        bool retire = false;
        if (j < k) {
            first = phrase_index_at(bitmap, tile_base, soff[j]);
            nextf = (j + 1 < k) ? phrase_index_at(bitmap, tile_base, soff[j + 1]) : P;
            retire = (nextf - first == 1);
        }
        u64 tot;
        u64 rb = block_excl_scan(retire ? 1ull : 0ull, tot) + carry;
        if (j < k) {
            if (retire) {
                R_phr[rb] = first;
                R_sid[rb] = sid[j];
            } else {
                soff_next[j - rb] = first - rb;
                sid_next[j - rb] = sid[j];
            }
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        soff_next[k - carry] = P - carry;
        rc->phrases = P;
        rc->retired = carry;
        rc->k_next = k - carry;
        rc->n_next = P - carry;
    }
}

// --------------------------------------------------------------------------
// k_phrases: fingerprints of phrases and phrase-table insertion
// --------------------------------------------------------------------------

// end (exclusive) of the phrase starting at `pos`: next set bit after pos, or n
__device__ u64 phrase_end(const u32* bitmap, u64 nw, u64 n, u64 pos) {
    u64 w = pos / 32;
    u32 bit = (u32)(pos & 31);
    u32 m = (bit == 31) ? 0u : (bitmap[w] & ~((2u << bit) - 1u));
    while (m == 0) {
        if (++w >= nw) return n;
        m = bitmap[w];
    }
    u64 e = w * 32 + (__ffs(m) - 1);
    return e < n ? e : n;
}

template <typename T>
__device__ bool same_content(const T* S, u64 ra, u64 rb, u64 len) {
    for (u64 x = 0; x < len; x++)
        if (S[ra + x] != S[rb + x]) return false;
    return true;
}

// Insert the phrase S[pos, pos+len) (phrase index pidx) and return its slot, or
// ~0u when the pass must stop (table over its load limit, or an error).
template <typename T>
__device__ u32 table_insert(Slot* tab, u64 mask, u64 claim_limit, u64 key, u64 pos, u64 len, u32 fpv, u64 pidx,
                            const T* S, const u32* bitmap, u64 nw, u64 n, DevStatus* ds) {
    u64 s = key_home(key) & mask;
    for (u64 probe = 0; probe <= mask; probe++) {
        Slot* sl = tab + s;
        u64 kk = ld_relaxed(&sl->key);
        u64 ref;
        if (kk == kEmpty) {
            if (vload(&ds->overflow)) return ~0u;
            u64 ok, oref;
            cas128(sl, kEmpty, kEmpty, key, pos, ok, oref);
            if (ok == kEmpty) {
                sl->len = (u32)len;
                sl->fp = fpv;
                atomicMin(&sl->minp, pidx);
                u64 c = atomicAdd(&ds->claims, 1ull);
                atomicAdd(&ds->claim_len, len);
                if (c + 1 > claim_limit) atomicExch(&ds->overflow, 1u);
                return (u32)s;
            }
            kk = ok;
            ref = oref;
        } else {
            ref = ld_relaxed(&sl->ref);
            u64 it = 0;
            while (ref == kEmpty) {  // the pair is written at once; guard only
                if (++it > kSpinLimit) { set_error(ds, kErrTimeout); return ~0u; }
                ref = ld_relaxed(&sl->ref);
            }
        }
        if (kk == key) {
            // saturated length field: check the stored phrase's length first
            bool ok = (len < kLenSat) || (phrase_end(bitmap, nw, n, ref) - ref == len);
            if (ok && same_content<T>(S, ref, pos, len)) {
                if (pidx < ld_relaxed(&sl->minp)) atomicMin(&sl->minp, pidx);
                return (u32)s;
            }
        }
        s = (s + 1) & mask;
    }
    set_error(ds, kErrTableFull);
    return ~0u;
}

// Rank of the phrase S[pos, pos+len) among the rules of a resident level
// (table rtab over the rules rrhs/rrhs_off), or ~0u when it is not one of them.
template <typename T>
__device__ u32 resident_find(const Slot* rtab, u64 rmask, const u32* rrhs, const u64* rrhs_off, u64 key,
                             const T* S, u64 pos, u64 len) {
    u64 s = key_home(key) & rmask;
    for (u64 probe = 0; probe <= rmask; probe++) {
        const u64 kk = rtab[s].key;
        if (kk == kEmpty) return ~0u;
        if (kk == key) {
            const u64 r = rtab[s].ref;
            const u64 o = rrhs_off[r];
            if (rrhs_off[r + 1] - o == len) {
                bool eq = true;
                for (u64 x = 0; x < len && eq; x++) eq = ((u32)S[pos + x] == rrhs[o + x]);
                if (eq) return (u32)r;
            }
        }
        s = (s + 1) & rmask;
    }
    return ~0u;
}

template <typename T>
__global__ void __launch_bounds__(kTileWords) k_phrases(const T* __restrict__ S, u64 n,
                                                        const u32* __restrict__ Fprev, LevelHash lh,
                                                        const u32* __restrict__ bitmap,
                                                        const u64* __restrict__ tile_base, Slot* tab, u64 mask,
                                                        u64 claim_limit, const Slot* __restrict__ rtab, u64 rmask,
                                                        const u32* __restrict__ rrhs,
                                                        const u64* __restrict__ rrhs_off,
                                                        u32* __restrict__ P_slot, DevStatus* ds) {
    __shared__ u32 sF[256];
    __shared__ unsigned short sStart[kTilePos];
    __shared__ u64 sTailEnd;
    FpSource<T> fp;
    if constexpr (sizeof(T) == 1) {
        for (int x = threadIdx.x; x < 256; x += blockDim.x) sF[x] = Fprev[x];
        fp.F = sF;
    } else {
        fp.F = Fprev;
    }
    const u64 tile = blockIdx.x;
    const u64 nw = (n + 31) / 32;
    const u64 w = tile * kTileWords + threadIdx.x;
    u32 word = (w < nw) ? bitmap[w] : 0u;
    u64 total;
    u64 off = block_excl_scan((u64)__popc(word), total);
    {
        u32 m = word;
        u32 o = (u32)off;
        while (m) {
            int b = __ffs(m) - 1;
            m &= m - 1;
            sStart[o++] = (unsigned short)(threadIdx.x * 32 + b);
        }
    }
    if (threadIdx.x == 0) {
        u64 tile_end = (tile + 1) * (u64)kTilePos;
        sTailEnd = (tile_end >= n) ? n : phrase_end(bitmap, nw, n, tile_end - 1);
    }
    __syncthreads();
    const u64 t0 = tile * (u64)kTilePos;
    const u64 pbase = tile_base[tile];
    for (u32 q = threadIdx.x; q < (u32)total; q += blockDim.x) {
        const u64 start = t0 + sStart[q];
        const u64 end = (q + 1 < (u32)total) ? t0 + sStart[q + 1] : sTailEnd;
        const u64 len = end - start;
        if (len >= (1ull << 32)) { set_error(ds, kErrPhraseLong); P_slot[pbase + q] = ~0u; continue; }
        // H = sum_j F[Q_j] c^{j-1} mod p, by Horner from the last symbol
        u64 H = 0;
        for (u64 x = end; x-- > start;) H = addmod61(mulmod61(H, lh.c), (u64)fp(S[x]));
        const u32 fpv = finish_hash(lh, H);
        const u64 key = make_key(H, len);
        if (rtab != nullptr) {
            const u32 r = resident_find<T>(rtab, rmask, rrhs, rrhs_off, key, S, start, len);
            if (r != ~0u) { P_slot[pbase + q] = kResidentBit | r; continue; }
        }
        P_slot[pbase + q] = table_insert<T>(tab, mask, claim_limit, key, start, len, fpv, pbase + q, S, bitmap,
                                            nw, n, ds);
    }
}

// --------------------------------------------------------------------------
// k_name: first-occurrence ranks, level-i rules and fingerprints
// --------------------------------------------------------------------------

// Claim a free slot of a resident table for rule `rank` with key `key` (rules
// of a level are distinct, so no comparison is needed).
__device__ void resident_insert(Slot* rtab, u64 rmask, u64 key, u64 rank, DevStatus* ds) {
    u64 s = key_home(key) & rmask;
    for (u64 probe = 0; probe <= rmask; probe++) {
        u64 ok, oref;
        cas128(rtab + s, kEmpty, kEmpty, key, rank, ok, oref);
        if (ok == kEmpty) return;
        s = (s + 1) & rmask;
    }
    set_error(ds, kErrTableFull);
}

template <typename T>
__global__ void __launch_bounds__(kNameThreads) k_name(const u32* __restrict__ P_slot, const u64* __restrict__ Pp,
                                                       Slot* tab, const T* __restrict__ S, u64 g_base, u64 G_base,
                                                       u32* __restrict__ rhs, u64* __restrict__ rhs_off,
                                                       u32* __restrict__ F, LBSlot<2>* lb, u64 epoch, u64* ctr,
                                                       u64 ctr_base, u64* __restrict__ totals, Slot* rtab_w,
                                                       u64 rmask_w, DevStatus* ds) {
    const u64 P = *Pp;
    const u64 tile = dynamic_tile(ctr, ctr_base);
    const u64 p0 = tile * (u64)kNameTile;
    if (p0 >= P) return;  // grid is sized from an upper bound of P
    u32 slot[kNameItems];
    bool first[kNameItems];
    u64 len[kNameItems];
    u64 cnt = 0, lsum = 0;
#pragma unroll
    for (int it = 0; it < kNameItems; it++) {
        const u64 p = p0 + (u64)threadIdx.x * kNameItems + it;  // blocked: keeps order
        first[it] = false;
        len[it] = 0;
        slot[it] = 0;
        if (p < P) {
            slot[it] = P_slot[p];
            if (!(slot[it] & kResidentBit)) {
                first[it] = (tab[slot[it]].minp == p);
                if (first[it]) len[it] = tab[slot[it]].len;
            }
        }
        cnt += first[it];
        lsum += len[it];
    }
    u64 tc, tl;
    u64 ec = block_excl_scan(cnt, tc);
    u64 el = block_excl_scan(lsum, tl);
    u64 agg[2] = {tc, tl}, excl[2];
    block_lookback<2>(lb, tile, epoch, agg, excl, ds);
    u64 r = g_base + excl[0] + ec;
    u64 o = G_base + excl[1] + el;
#pragma unroll
    for (int it = 0; it < kNameItems; it++) {
        if (!first[it]) continue;
        Slot* sl = tab + slot[it];
        const u64 ref = sl->ref;
        F[r] = sl->fp;
        rhs_off[r] = o;
        for (u64 x = 0; x < len[it]; x++) rhs[o + x] = (u32)S[ref + x];
        sl->ref = r;  // the slot now names its rank
        if (rtab_w != nullptr) resident_insert(rtab_w, rmask_w, sl->key, r, ds);
        r++;
        o += len[it];
    }
    if (p0 + kNameTile >= P && threadIdx.x == 0) {
        const u64 g_end = g_base + excl[0] + tc, G_end = G_base + excl[1] + tl;
        rhs_off[g_end] = G_end;
        totals[0] = g_end;
        totals[1] = G_end;
    }
}

// --------------------------------------------------------------------------
// k_rewrite: T^{i+1} and retired strings
// --------------------------------------------------------------------------

__global__ void k_rewrite(const u32* __restrict__ P_slot, const u64* __restrict__ Pp, const Slot* __restrict__ tab,
                          u32* __restrict__ Tnext, const u64* __restrict__ R_phr, const u32* __restrict__ R_sid,
                          const RoundCounts* __restrict__ rc, u32 level, u32* __restrict__ c_level,
                          u32* __restrict__ c_rank) {
    const u64 P = *Pp;
    const u64 nr = rc->retired;
    for (u64 p = blockIdx.x * (u64)blockDim.x + threadIdx.x; p < P; p += (u64)gridDim.x * blockDim.x) {
        const u32 s = P_slot[p];
        const u32 r = (s == ~0u) ? 0u : ((s & kResidentBit) ? (s & ~kResidentBit) : (u32)tab[s].ref);
        if (nr == 0) { Tnext[p] = r; continue; }
        u64 lo = 0, hi = nr;  // first index with R_phr >= p
        while (lo < hi) {
            u64 mid = (lo + hi) >> 1;
            if (R_phr[mid] < p) lo = mid + 1; else hi = mid;
        }
        if (lo < nr && R_phr[lo] == p) {
            c_level[R_sid[lo]] = level;
            c_rank[R_sid[lo]] = r;
        } else {
            Tnext[p - lo] = r;
        }
    }
}

// --------------------------------------------------------------------------
// k_resident_build: table over the existing rules of a level
// --------------------------------------------------------------------------

// Rules r0 .. r0+cnt-1 of a level enter its resident table.
__global__ void k_resident_build(const u32* __restrict__ rhs, const u64* __restrict__ rhs_off, u64 r0, u64 cnt,
                                 const u32* __restrict__ Fprev, LevelHash lh, Slot* rtab, u64 rmask, DevStatus* ds) {
    for (u64 x = blockIdx.x * (u64)blockDim.x + threadIdx.x; x < cnt; x += (u64)gridDim.x * blockDim.x) {
        const u64 r = r0 + x;
        const u64 s = rhs_off[r], e = rhs_off[r + 1];
        u64 H = 0;
        for (u64 y = e; y-- > s;) H = addmod61(mulmod61(H, lh.c), (u64)__ldg(Fprev + rhs[y]));
        resident_insert(rtab, rmask, make_key(H, e - s), r, ds);
    }
}

// --------------------------------------------------------------------------
// round 0 helpers: strings of length one, and gathering the active strings
// --------------------------------------------------------------------------

__global__ void k_level0(const unsigned char* __restrict__ data, const u64* __restrict__ pos,
                         const u32* __restrict__ ids, u32 cnt, u32* c_level, u32* c_rank) {
    u32 x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < cnt) {
        c_level[ids[x]] = 0;
        c_rank[ids[x]] = data[pos[x]];
    }
}

__global__ void k_gather_strings(const unsigned char* __restrict__ data, const u64* __restrict__ src_off,
                                 const u64* __restrict__ dst_off, u32 k, unsigned char* __restrict__ out) {
    for (u32 j = blockIdx.x; j < k; j += gridDim.x) {
        const u64 s = src_off[j], d = dst_off[j], len = dst_off[j + 1] - dst_off[j];
        for (u64 x = threadIdx.x; x < len; x += blockDim.x) out[d + x] = data[s + x];
    }
}

// --------------------------------------------------------------------------
// host launchers
// --------------------------------------------------------------------------

u64 tiles_for(u64 n) { return (n + kTilePos - 1) / kTilePos; }
u64 name_tiles_for(u64 P) { return (P + kNameTile - 1) / kNameTile; }

template <typename T>
static cudaError_t launch_breaks_t(const RoundArgs& a, cudaStream_t st) {
    const u64 tiles = tiles_for(a.n);
    k_breaks<T><<<(unsigned)tiles, kTileWords, 0, st>>>((const T*)a.S, a.n, a.soff, a.k, a.Fprev, a.bitmap,
                                                      a.tile_base, (LBSlot<1>*)a.lb1, a.epoch, a.ctr, a.ctr_base,
                                                      a.total, a.ds);
    return cudaGetLastError();
}

cudaError_t launch_breaks(const RoundArgs& a, cudaStream_t st) {
    return a.sym_bytes == 1 ? launch_breaks_t<unsigned char>(a, st) : launch_breaks_t<u32>(a, st);
}

cudaError_t launch_strings(const RoundArgs& a, cudaStream_t st) {
    k_strings<<<1, 1024, 0, st>>>(a.soff, a.sid, a.k, a.bitmap, a.tile_base, a.total, a.soff_next, a.sid_next,
                                  a.R_phr, a.R_sid, a.rc);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_phrases_t(const RoundArgs& a, cudaStream_t st) {
    const u64 tiles = tiles_for(a.n);
    k_phrases<T><<<(unsigned)tiles, kTileWords, 0, st>>>((const T*)a.S, a.n, a.Fprev, a.lh, a.bitmap, a.tile_base,
                                                       (Slot*)a.tab, a.mask, a.claim_limit, (const Slot*)a.rtab,
                                                       a.rmask, a.rrhs, a.rrhs_off, a.P_slot, a.ds);
    return cudaGetLastError();
}

cudaError_t launch_phrases(const RoundArgs& a, cudaStream_t st) {
    return a.sym_bytes == 1 ? launch_phrases_t<unsigned char>(a, st) : launch_phrases_t<u32>(a, st);
}

template <typename T>
static cudaError_t launch_name_t(const RoundArgs& a, cudaStream_t st) {
    const u64 tiles = name_tiles_for(a.P);
    if (tiles == 0) return cudaSuccess;
    k_name<T><<<(unsigned)tiles, kNameThreads, 0, st>>>(a.P_slot, a.total, (Slot*)a.tab, (const T*)a.S, a.g_base,
                                                       a.G_base, a.rhs, a.rhs_off, a.F, (LBSlot<2>*)a.lb2,
                                                       a.epoch, a.ctr, a.ctr_base, a.totals, (Slot*)a.rtab_w,
                                                       a.rmask_w, a.ds);
    return cudaGetLastError();
}

cudaError_t launch_name(const RoundArgs& a, cudaStream_t st) {
    return a.sym_bytes == 1 ? launch_name_t<unsigned char>(a, st) : launch_name_t<u32>(a, st);
}

cudaError_t launch_rewrite(const RoundArgs& a, cudaStream_t st) {
    u64 blocks = (a.P + 255) / 256;
    if (blocks == 0) return cudaSuccess;
    if (blocks > 152ull * 64) blocks = 152ull * 64;
    k_rewrite<<<(unsigned)blocks, 256, 0, st>>>(a.P_slot, a.total, (const Slot*)a.tab, a.Tnext, a.R_phr, a.R_sid,
                                                a.rc, a.level, a.c_level, a.c_rank);
    return cudaGetLastError();
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
    unsigned blocks = k < 152 * 8 ? k : 152 * 8;
    k_gather_strings<<<blocks, 256, 0, st>>>(data, src_off, dst_off, k, out);
    return cudaGetLastError();
}

cudaError_t launch_resident_build(const u32* rhs, const u64* rhs_off, u64 r0, u64 cnt, const u32* Fprev,
                                  LevelHash lh, void* rtab, u64 rmask, DevStatus* ds, cudaStream_t st) {
    if (cnt == 0) return cudaSuccess;
    u64 blocks = (cnt + 255) / 256;
    if (blocks > 152ull * 32) blocks = 152ull * 32;
    k_resident_build<<<(unsigned)blocks, 256, 0, st>>>(rhs, rhs_off, r0, cnt, Fprev, lh, (Slot*)rtab, rmask, ds);
    return cudaGetLastError();
}

size_t lb1_bytes(u64 tiles) { return tiles * sizeof(LBSlot<1>); }
size_t lb2_bytes(u64 tiles) { return tiles * sizeof(LBSlot<2>); }
size_t slot_bytes() { return sizeof(Slot); }

}  // namespace lcg
