// Content-addressed phrase tables (one per level and round).
//
// A table maps the content of a phrase (a sequence of level-(i-1) symbols) to
// a value: during a round's parse the value is the smallest phrase index among
// the phrase's occurrences, which decides first-occurrence naming; in the
// table of a resident grammar it is the rule's rank.
//
// Keys are 128 bits.  Short phrases are stored exactly ("inline" keys): the
// top 4 bits of `hi` hold the length q, and the symbols are packed from bit 0
// upwards in the 124 bits left, w bits each (8 for bytes; for ranks the width
// of the level below, at most 31), so q <= min(14, 124 / w).  Two inline keys
// of one width are equal exactly when the phrases are.  The length field is
// at most 14, so no key has hi == ~0, the mark of an empty slot (tables are
// cleared to all ones): with 15 bytes a phrase of 0xFF bytes would have
// packed to exactly that mark.  A longer phrase gets a "hashed" key: top 4
// bits 0, its length in bits 32..59 of `hi` and a 32-bit hash below, with `lo`
// naming where its content can be read; a hashed-key match is confirmed by
// comparing the contents symbol by symbol.  Slots are claimed with one 128-bit compare-and-swap.
// The home slot is the high half of mix(key) * cap, so any capacity works;
// the polynomial fingerprint H = sum_j F[Q_j] c^{j-1} mod p of a phrase is
// only needed for hashed keys.
#pragma once

#include "lcg_dev.cuh"

namespace lcg {

struct __align__(16) Key128 {
    u64 lo, hi;
};

// A slot holds its 128-bit key and its 64-bit value in one 32-byte sector, so
// that a lookup and the update of the value touch one sector.
struct __align__(32) Slot {
    Key128 key;
    u64 val;
    u64 spare;
};
static_assert(sizeof(Slot) == 32, "one sector per slot");

struct ContentTable {
    Slot* slots;
    u64 cap;  // 0: no table
};

constexpr u64 kEmptyHi = ~0ull;
constexpr int kHiBits = 60;
constexpr u64 kMaxPhraseLen = (1ull << 28) - 1;  // longest phrase a hashed key can describe

// Bits per symbol in inline keys: 8 for bytes; for ranks a width w with every
// rank of the level below < 2^w.  A round's own table uses the smallest such w
// (so that more phrases fit inline); tables that outlive a round (resident
// grammars, merges) use kRankBits.
constexpr int kRankBits = 31;
constexpr int kInlineMax = 14;
__device__ __forceinline__ u64 inline_max(int w) {
    const int m = 124 / w;
    return m < kInlineMax ? (u64)m : (u64)kInlineMax;
}

__device__ __forceinline__ void put_bits(u64& hi, u64& lo, int pos, u64 v, int b) {
    if (pos + b <= kHiBits) {
        hi |= v << pos;
    } else if (pos >= kHiBits) {
        lo |= v << (pos - kHiBits);
    } else {
        hi |= (v << pos) & ((1ull << kHiBits) - 1);
        lo |= v >> (kHiBits - pos);
    }
}

__device__ __forceinline__ u64 get_bits(u64 hi, u64 lo, int pos, int b) {
    const u64 m = (1ull << b) - 1;
    if (pos + b <= kHiBits) return (hi >> pos) & m;
    if (pos >= kHiBits) return (lo >> (pos - kHiBits)) & m;
    const u64 low = (hi >> pos) & ((1ull << (kHiBits - pos)) - 1);
    return (low | (lo << (kHiBits - pos))) & m;
}

// The inline key of get(0..len-1): the symbols form the number
// V = sum_j get(j) 2^(j b) (at most 124 bits), accumulated from the last
// symbol with a 128-bit shift per symbol (no branch on where a symbol falls);
// bits 0..59 of V go to hi under the length, bits 60..123 to lo.  This is the
// layout put_bits / key_sym use.
template <typename Get>
__device__ __forceinline__ Key128 key_inline(Get get, u64 len, int b) {
    u64 vlo = 0, vhi = 0;  // V, 128 bits
    for (u64 j = len; j-- > 0;) {
        vhi = (vhi << b) | (vlo >> (64 - b));  // b in 1..31: both shifts defined
        vlo = (vlo << b) | (u64)get(j);
    }
    const u64 hi = (len << kHiBits) | (vlo & ((1ull << kHiBits) - 1));
    const u64 lo = (vlo >> kHiBits) | (vhi << (64 - kHiBits));
    return Key128{lo, hi};
}

__device__ __forceinline__ Key128 key_hashed(u64 H, u64 len, u64 ref) {
    const u32 h = (u32)fmix64(H ^ (len * 0x9E3779B97F4A7C15ull));
    return Key128{ref, (len << 32) | (u64)h};
}

__device__ __forceinline__ bool key_is_hashed(const Key128& k) { return (k.hi >> kHiBits) == 0; }

__device__ __forceinline__ u64 key_len(const Key128& k) {
    const u64 l = k.hi >> kHiBits;
    return l ? l : ((k.hi >> 32) & kMaxPhraseLen);
}

// symbol j of an inline key
__device__ __forceinline__ u32 key_sym(const Key128& k, u64 j, int b) {
    return (u32)get_bits(k.hi, k.lo, (int)j * b, b);
}

// Home slot of a key: the high half of mix(key) * cap.  An inline key is the
// content itself; a hashed key's high half carries the length and a hash of
// the phrase's fingerprint (its low half names a location, not content).  The
// mix is a multiply-xorshift of both halves (two 64-bit products).
__device__ __forceinline__ u64 key_home(const Key128& k, u64 cap) {
    const u64 lo = key_is_hashed(k) ? 0ull : k.lo;
    u64 m = (lo ^ (k.hi * 0x9E3779B97F4A7C15ull)) * 0xD6E8FEB86659FD93ull;
    m ^= m >> 32;
    return __umul64hi(m, cap);
}

__device__ __forceinline__ Key128 ld_key_relaxed(const Key128* p) {
    Key128 k;
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(k.lo), "=l"(k.hi) : "l"(p) : "memory");
    return k;
}

// A slot's key and value with one 32-byte load (one request for the sector).
// The two halves need not be read at one instant: the key is checked as
// before, and the value is only used as an upper bound of the stored value,
// which never increases.
__device__ __forceinline__ Key128 ld_slot_relaxed(const Slot* p, u64* val) {
    Key128 k;
    u64 spare;
    asm volatile("ld.relaxed.gpu.global.v4.u64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(k.lo), "=l"(k.hi), "=l"(*val), "=l"(spare)
                 : "l"(p)
                 : "memory");
    (void)spare;
    return k;
}

__device__ __forceinline__ Key128 cas_key(Key128* p, Key128 cmp, Key128 val) {
    Key128 old;
    asm volatile(
        "{\n\t"
        ".reg .b128 c, n, d;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 n, {%4, %5};\n\t"
        "atom.relaxed.gpu.global.cas.b128 d, [%6], c, n;\n\t"
        "mov.b128 {%0, %1}, d;\n\t"
        "}"
        : "=l"(old.lo), "=l"(old.hi)
        : "l"(cmp.lo), "l"(cmp.hi), "l"(val.lo), "l"(val.hi), "l"(p)
        : "memory");
    return old;
}

// Longest probe sequence of a claim: far beyond what a table under its load
// limit shows, so reaching it means the table is (nearly) full.
constexpr u64 kMaxProbes = 4096;
// Slots read together (G, a power of two up to 4: at most one 128-byte line):
// the rest of the home slot's group of G, then whole groups.  A warp waits for
// its longest probe sequence, and a group costs one round trip instead of one
// per slot.

// Find or claim the slot of key k in a table that other threads are filling.
// `same(ref)` compares the content stored at `ref` with the phrase (hashed keys
// only).  The slot's value is lowered to `pidx` (first occurrence).  Returns
// the slot and sets *claimed when this call claimed it, or ~0 when the table
// is over its load limit or full, or the probe sequence reached kMaxProbes
// (the host then regrows the table and reruns).  Slots are examined in probe
// order, and a new key goes into the first empty one: a slot read as empty may
// have been claimed since (the compare-and-swap then returns its key), but one
// read as taken stays so, as keys are never removed.
template <int G, typename Same>
__device__ u64 table_claim_or_find(ContentTable t, const Key128& k, bool hashed, u64 pidx, Same same, bool* claimed,
                                   DevStatus* ds) {
    static_assert(G == 1 || G == 2 || G == 4, "groups of 1, 2 or 4 slots");
    u64 s = key_home(k, t.cap);
    const Key128 empty{~0ull, ~0ull};
    const u64 limit = t.cap < kMaxProbes ? t.cap : kMaxProbes;
    u32 groups = 0;
    for (u64 probe = 0; probe < limit;) {
        // once the table is over its load limit the pass is rerun: stop early
        if ((++groups & 15) == 0 && vload(&ds->overflow)) return ~0ull;
        const u64 gend = min((s | (u64)(G - 1)) + 1, t.cap);
        const int m = (int)min(gend - s, limit - probe);
        // every slot of the group whole (key and value, one request each): a
        // found key whose value is already at most pidx needs no update
        Key128 c[G];
        u64 cv[G];
#pragma unroll
        for (int j = 0; j < G; j++)
            if (j < m) c[j] = ld_slot_relaxed(&t.slots[s + j], &cv[j]);
#pragma unroll
        for (int j = 0; j < G; j++) {
            if (j >= m) break;
            Key128* kp = &t.slots[s + j].key;
            Key128 cur = c[j];
            if (cur.hi == kEmptyHi) {
                const Key128 old = cas_key(kp, empty, k);
                if (old.hi == kEmptyHi) {
                    *claimed = true;
                    atomicMin(&t.slots[s + j].val, pidx);
                    return s + j;
                }
                cur = old;
                cv[j] = ~0ull;  // read before the slot was claimed
            }
            if (cur.hi == k.hi) {
                // a pair read while being written shows the empty low half: read it again atomically
                if (cur.lo == ~0ull) cur = cas_key(kp, empty, empty);
                if (hashed ? same(cur.lo) : (cur.lo == k.lo)) {
                    if (cv[j] > pidx) atomicMin(&t.slots[s + j].val, pidx);  // values only decrease
                    return s + j;
                }
            }
        }
        probe += (u64)m;
        s = (gend == t.cap) ? 0 : gend;
    }
    atomicExch(&ds->overflow, 1u);
    return ~0ull;
}

// table_claim_or_find by a whole warp for one hashed key (a long phrase): every
// lane calls it with the same arguments.  Lane 0 reads and claims the slots, in
// the same probe order as table_claim_or_find (so both find a key wherever the
// other put it); `same(ref)` is a warp-wide content comparison run by all lanes.
// Every lane returns the slot and *claimed.
template <typename SameWarp>
__device__ u64 table_claim_or_find_warp(ContentTable t, const Key128& k, u64 pidx, SameWarp same, bool* claimed,
                                        DevStatus* ds) {
    const u32 lane = threadIdx.x & 31;
    u64 s = key_home(k, t.cap);
    const Key128 empty{~0ull, ~0ull};
    const u64 limit = t.cap < kMaxProbes ? t.cap : kMaxProbes;
    *claimed = false;
    for (u64 probe = 0; probe < limit; probe++) {
        Key128 cur{0, 0};
        int took = 0, stop = 0;
        if (lane == 0) {
            if ((probe & 15) == 15 && vload(&ds->overflow)) stop = 1;
            Key128* kp = &t.slots[s].key;
            cur = ld_key_relaxed(kp);
            if (!stop && cur.hi == kEmptyHi) {
                const Key128 old = cas_key(kp, empty, k);
                if (old.hi == kEmptyHi) {
                    took = 1;
                    atomicMin(&t.slots[s].val, pidx);
                }
                cur = old;
            }
            if (!stop && !took && cur.hi == k.hi && cur.lo == ~0ull) cur = cas_key(kp, empty, empty);
        }
        stop = __shfl_sync(0xffffffffu, stop, 0);
        if (stop) return ~0ull;
        took = __shfl_sync(0xffffffffu, took, 0);
        if (took) {
            *claimed = true;
            return s;
        }
        cur.lo = __shfl_sync(0xffffffffu, cur.lo, 0);
        cur.hi = __shfl_sync(0xffffffffu, cur.hi, 0);
        if (cur.hi == k.hi && same(cur.lo)) {
            if (lane == 0) atomicMin(&t.slots[s].val, pidx);
            return s;
        }
        s = (s + 1 == t.cap) ? 0 : s + 1;
    }
    if (lane == 0) atomicExch(&ds->overflow, 1u);
    return ~0ull;
}

// table_find by a whole warp for one hashed key; `same(lo)` is a warp-wide
// comparison.  Every lane returns the value, or ~0 when absent.
template <typename SameWarp>
__device__ u64 table_find_warp(const ContentTable& t, const Key128& k, SameWarp same) {
    u64 s = key_home(k, t.cap);
    for (u64 probe = 0; probe < t.cap; probe++) {
        const Key128 cur = t.slots[s].key;  // the same address on every lane
        if (cur.hi == kEmptyHi) return ~0ull;
        if (cur.hi == k.hi && same(cur.lo)) return t.slots[s].val;
        s = (s + 1 == t.cap) ? 0 : s + 1;
    }
    return ~0ull;
}

// Look a key up in a table that nobody writes during the call.  `same(lo)`
// confirms hashed keys.  Returns the slot's value, or ~0 when absent.
template <typename Same>
__device__ u64 table_find(const ContentTable& t, const Key128& k, bool hashed, Same same) {
    u64 s = key_home(k, t.cap);
    for (u64 probe = 0; probe < t.cap; probe++) {
        const Key128 cur = t.slots[s].key;
        if (cur.hi == kEmptyHi) return ~0ull;
        if (cur.hi == k.hi && (hashed ? same(cur.lo) : (cur.lo == k.lo))) return t.slots[s].val;
        s = (s + 1 == t.cap) ? 0 : s + 1;
    }
    return ~0ull;
}

// Claim a free slot for a key known to be absent (rules of a level are
// distinct) and store `val`.
__device__ __forceinline__ void table_put(ContentTable t, const Key128& k, u64 val, DevStatus* ds) {
    u64 s = key_home(k, t.cap);
    const Key128 empty{~0ull, ~0ull};
    for (u64 probe = 0; probe < t.cap; probe++) {
        const Key128 old = cas_key(&t.slots[s].key, empty, k);
        if (old.hi == kEmptyHi) {
            t.slots[s].val = val;
            return;
        }
        s = (s + 1 == t.cap) ? 0 : s + 1;
    }
    set_error(ds, kErrTableFull);
}

// Key of a rule of level `level` whose right-hand side is get(0..len-1)
// (bytes at level 1), with polynomial fingerprint H, for a table whose values
// are ranks: hashed keys name the rank.
template <typename Get>
__device__ __forceinline__ Key128 rule_key(Get get, u64 len, int w, u64 H, u64 rank) {
    if (len <= inline_max(w)) return key_inline(get, len, w);
    return key_hashed(H, len, rank);
}

}  // namespace lcg
