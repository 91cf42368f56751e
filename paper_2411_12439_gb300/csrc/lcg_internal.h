// Host-side declarations shared by the translation units of the library
// (launchers of the kernels and the argument blocks they take).
#pragma once

#include <cstddef>
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>
#include <utility>

#include "lcg_dev.cuh"

namespace lcg {

// Launch of a kernel that starts with pdl_wait(), with programmatic dependent
// launch allowed (also inside stream capture, where it becomes a programmatic
// edge of the graph).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// A cooperative launch (every block resident at once: the kernel's blocks
// may wait for one another), with programmatic dependent launch like the
// others (the kernel's first steps wait for the grid before it).
template <typename... KArgs, typename... Args>
cudaError_t launch_coop(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Counts written by k_strings for the host.
struct RoundCounts {
    u64 phrases;  // phrases of the round (= |T^{i+1}| before retiring)
    u64 retired;  // strings that became one symbol
    u64 k_next;   // strings still active
    u64 n_next;   // |T^{i+1}|
    u64 tiles;    // parse tiles of the round
    u64 pad[3];
};

struct RoundArgs {
    int sym_bytes;        // 1 in round 1 (bytes), 4 afterwards (ranks)
    int sym_w;            // bits per symbol in the round's inline keys (every symbol < 2^sym_w)
    const void* S;        // T^i
    const u32* Sf;        // fingerprints of T^i (rounds >= 2)
    u64 n;                // |T^i| (when d_n is null)
    const u64* d_n;       // |T^i| on the device (rounds enqueued without a host sync), or null
    const u64* soff;      // k+1 string offsets into T^i
    const u32* sid;       // original string index of each active string
    u32 k;                // active strings (when d_k is null)
    const u64* d_k;       // active strings on the device, or null
    const u32* Fprev;     // F^{i-1}
    LevelHash lh;         // parameters of h^i
    u32 level;            // i
    u32 parse_blocks;     // resident k_parse blocks per SM (0: as many as fit)
    u32 stripes;          // rounds >= 2: tiles taken in this many interleaved stripes (1: in order)
    u32 miss_flush;       // byte rounds: queued cache misses that trigger a lookup pass
    u32 tp;               // positions per parse tile (1024, 2048 or 4096): order keys are tile * tp + q
    // parse pass
    u64 tiles_bound;      // parse tiles the buffers were sized for
    u64* d_tiles;         // parse tiles of the round (written by k_tile_strings)
    u32* brk;             // break bitmap of T^i (k_breaks), 64 words per parse tile
    u32* sbm;             // bitmap of string starts of T^i (and of n)
    u64 sbm_words;
    u32* tile_str;        // per parse tile: the string holding its first position
    u32* tile_cnt;        // per parse tile: phrases starting in it
    u64* tile_pfx;        // exclusive prefix of tile_cnt: global index of a tile's first phrase
    u64* string_first;    // order key (tile * TP + q) of each active string's first phrase
    void* lb1;            // look-back slots
    u64 epoch;
    u64* heads;           // k_breaks: the head word of each block step (its own buffer)
    u64 brk_epoch;        // epoch of k_breaks' head words
    u64* ctr;
    u64 ctr_base;
    u64* total;           // device: phrases of the round
    DevStatus* ds;
    void* tab;            // the round's phrase table (32-byte slots)
    u64 tab_cap;
    u64 claim_limit;
    u32* claims;          // slots claimed in this round (tab_cap entries)
    void* rtab;           // table of the resident level i (read), or cap 0
    u64 rtab_cap;
    const u32* rrhs;
    const u64* rrhs_off;
    u32* P_slot;          // per phrase (tile t's phrases from pslot_base(t) on): slot, or a
                          // resident rank with the top bit set
    // strings pass
    u64* soff_next;
    u32* sid_next;
    u64* R_phr;
    u32* R_sid;
    RoundCounts* rc;
    const DevStatus* ds_prev;  // status of the round before (rounds enqueued without a sync), or null
    // naming pass
    const u64* d_gnew;    // new rules of the round (device: the claim count)
    const u64* d_Gnew;    // their total length (device)
    u64 g_alloc;          // entries of slot_r, len_r, xlen
    u64 cap_g, cap_G;     // capacity of the level's arrays
    u32* first_bits;      // bitmap over phrase indices
    u32* first_prefix;    // exclusive popcount prefix of its words
    u32* slot_r;          // slot of the rank-r new rule
    u32* len_r;           // its length
    void* mkey;           // claim c: its slot's key (Key128), read once by k_mark
    u64* mval;            // claim c: its slot's value (first occurrence)
    void* rkey;           // key of the rank-r new rule (Key128), for k_rules
    u64* rv;              // per table slot: (F^i << 32) | rank of its rule (k_rules, read by k_rewrite)
    u64* xlen;            // exclusive prefix of len_r
    u64 g_base, G_base;   // rules / rhs symbols of level i before this round

    u32* rhs;
    u64* rhs_off;
    u32* F;
    void* rtab_w;         // table of level i to extend with the new rules, or cap 0
    u64 rtab_w_cap;
    // rewrite pass
    u64 T_cap;            // entries of Tnext / Fnext
    u32* Tnext;
    u32* Fnext;           // fingerprints of T^{i+1}
    u32* c_level;
    u32* c_rank;
};

constexpr double kL2Bytes = 126.5 * 1024 * 1024;  // GB300 L2 (byte accounting, launch choices)
bool parse_tile_valid(u32 tp);                 // 1024, 2048 or 4096 positions
bool round_is_small(const RoundArgs& a);        // the round runs as k_parse_small and k_naming_small
u32 small_round_grid(const RoundArgs& a);       // their blocks (one launch of each per round)
constexpr u32 kSmallParseBarriers = 3, kSmallNamingBarriers = 5;  // grid barriers of each
u64 parse_slot_entries(u64 tiles, u64 strings, u32 tp);  // entries of P_slot for a round's tiles and strings
u64 breaks_steps(u64 tiles, u32 tp);                     // k_breaks' block steps over a round's parse tiles
u64 popscan_tiles_for(u64 nw);
size_t lb1_bytes(u64 tiles);
size_t lb2_bytes(u64 tiles);
size_t slot_bytes();  // bytes of one phrase-table slot

cudaError_t launch_tile_strings(const RoundArgs& a, cudaStream_t st);
cudaError_t launch_breaks(const RoundArgs& a, cudaStream_t st);
cudaError_t launch_parse(const RoundArgs& a, cudaStream_t st);
cudaError_t launch_parse_small(const RoundArgs& a, u64 bar_base, cudaStream_t st);
cudaError_t launch_naming_small(const RoundArgs& a, u64 nw, u64 g_bound, u64 bar_base, cudaStream_t st);
int parse_max_blocks(int sym_bytes);  // resident k_parse blocks per SM at most
cudaError_t launch_strings(const RoundArgs& a, cudaStream_t st);
cudaError_t launch_mark(const RoundArgs& a, u64 g_grid, cudaStream_t st);
cudaError_t launch_popscan(const RoundArgs& a, u64 nw_bound, cudaStream_t st);
cudaError_t launch_rank(const RoundArgs& a, u64 g_grid, cudaStream_t st);
cudaError_t launch_rules(const RoundArgs& a, u64 g_grid, cudaStream_t st);
cudaError_t launch_rewrite(const RoundArgs& a, cudaStream_t st);
cudaError_t launch_level0(const unsigned char* data, const u64* pos, const u32* ids, u32 cnt, u32* c_level,
                          u32* c_rank, cudaStream_t st);
cudaError_t launch_resident_build(const u32* rhs, const u64* rhs_off, u64 r0, u64 cnt, bool bytes, const u32* Fprev,
                                  LevelHash lh, void* slots, u64 cap, DevStatus* ds, cudaStream_t st);
cudaError_t launch_h0(LevelHash h0, u32* F0, cudaStream_t st);
cudaError_t launch_gather_strings(const unsigned char* data, const u64* src_off, const u64* dst_off, u32 k,
                                  unsigned char* out, cudaStream_t st);

// grammar.cu
cudaError_t launch_remap(const u32* in, u64 n, const u32* M, u32* out, cudaStream_t st);
cudaError_t launch_merge_lookup(const u32* brhs, const u64* brhs_off, const u32* bF, u64 gb, bool bytes,
                                const u32* aFprev, LevelHash lh, void* aslots, u64 acap, const u32* arhs,
                                const u64* arhs_off, const u32* aF, u32* M, u32* miss, u32* mlen, DevStatus* ds,
                                cudaStream_t st);
cudaError_t launch_merge_append(const u32* brhs, const u64* brhs_off, const u32* bF, u64 gb, const u32* miss,
                                const u64* xrank, const u64* xlen, u64 ga, u64 Ga, u32* arhs, u64* arhs_off,
                                u32* aF, u32* M, u64 ga_new, u64 Ga_new, cudaStream_t st);
cudaError_t launch_check_fp(const u32* rhs, const u64* rhs_off, u64 g, const u32* Fprev, LevelHash lh, const u32* F,
                            DevStatus* ds, cudaStream_t st);
// F arrays of a grammar by level (F[0] = F^0).
struct FTable {
    const u32* F[65];
    u32 n;
};
cudaError_t launch_roots(const u32* c_level, const u32* c_rank, u32 j0, u32 cnt, const FTable& ft, u32* out,
                         cudaStream_t st);
cudaError_t launch_remap_c(const u32* c_level, u32* c_rank, u32 k, u32 level, const u32* M, cudaStream_t st);
cudaError_t launch_rule_lens(const u32* cur, u64 cnt, const u64* rhs_off, u32* lens, cudaStream_t st);
cudaError_t launch_expand(const u32* cur, u64 cnt, const u64* offs, const u64* rhs_off, const u32* rhs, u32* next,
                          cudaStream_t st);
cudaError_t launch_to_bytes(const u32* cur, u64 cnt, unsigned char* out, cudaStream_t st);
// Exclusive scan of n elements; when n_dev is given the count is min(*n_dev, n)
// read on the device (n then only bounds the grid).
cudaError_t launch_scan2(const u32* in0, const u32* in1, u64 n, u64* out0, u64* out1, u64* totals, void* lb,
                         u64 epoch, u64* ctr, u64 ctr_base, DevStatus* ds, cudaStream_t st, u64* grid_out,
                         const u64* n_dev = nullptr);
u64 scan2_tiles_for(u64 n);
size_t scan2_lb_bytes(u64 tiles);
constexpr size_t scan2_lb_bytes_static(u64 tiles) { return tiles * sizeof(LBSlot<2>); }

// Post-processing (post.cu): the RL-rewritten levels of a grammar and what
// Simp decides about their rules.  Passed by value to the kernels.
constexpr int kPPMaxLevels = 64;
struct PPLevels {
    u32 n;                          // levels
    const u64* off[kPPMaxLevels];   // RL-rewritten right-hand-side offsets (g + 1)
    const u32* rhs[kPPMaxLevels];   // RL-rewritten right-hand sides (symbol, or 2^31 | run-length rule)
    u64 g[kPPMaxLevels];            // rules of the level
    u64 nrl[kPPMaxLevels];          // run-length rules of the level
    const u32* rl_y[kPPMaxLevels];  // their base symbol (of the level below)
    const u32* rl_l[kPPMaxLevels];  // and run length
    u8* pinned[kPPMaxLevels];       // the rule is a string's root or a run-length rule's base
    const u32* surv[kPPMaxLevels];  // the rule survives Simp
    const u64* spre[kPPMaxLevels];  // exclusive prefix of surv
    u32* explen[kPPMaxLevels];      // right-hand-side length with the removed rules below expanded
    u64* dst[kPPMaxLevels];         // output position of a removed rule's expansion
    u64 base[kPPMaxLevels];         // output id of the level's first surviving rule
    u64 S[kPPMaxLevels];            // surviving rules of the level
};

cudaError_t launch_rl_count(const u64* off, const u32* rhs, u64 g, u32* out_len, u32* rl_len, cudaStream_t st);
cudaError_t launch_rl_write(const u64* off, const u32* rhs, u64 g, const u64* new_off, const u64* rl_off, u32* new_rhs,
                            u32* run_y, u32* run_len, u64* run_pos, u64* keys, u64* vals, u64 mask, DevStatus* ds,
                            cudaStream_t st);
cudaError_t launch_rl_first(const u32* run_y, const u32* run_len, u64 R, const u64* keys, const u64* vals, u64 mask,
                            u32* first, u64* run_first, DevStatus* ds, cudaStream_t st);
cudaError_t launch_rl_fix(const u32* run_y, const u32* run_len, const u64* run_pos, const u64* run_first,
                          const u64* rank_of, u64 R, u32* new_rhs, u32* rl_y, u32* rl_l, DevStatus* ds,
                          cudaStream_t st);
cudaError_t launch_pp_uses(const u64* off, const u32* rhs, u64 g, u32* uses_below, cudaStream_t st);
cudaError_t launch_pp_pin_bases(const u32* rl_y, u64 nrl, u8* pinned_below, cudaStream_t st);
cudaError_t launch_pp_pin_roots(const u32* c_level, const u32* c_rank, u32 k, const PPLevels& lv, cudaStream_t st);
cudaError_t launch_pp_survive(const u32* uses, const u8* pinned, u64 g, u32* surv, cudaStream_t st);
cudaError_t launch_pp_lengths(const PPLevels& lv, u32 li, u32* fin_len, DevStatus* ds, cudaStream_t st);
cudaError_t launch_pp_write(const PPLevels& lv, u32 li, const u64* fin_off, u32* out, u8* kind, DevStatus* ds,
                            cudaStream_t st);
cudaError_t launch_pp_roots(const u32* c_level, const u32* c_rank, u32 k, const PPLevels& lv, u32* c_out,
                            cudaStream_t st);

// VByte codec (vbyte.cu).  A column is a u32 array (`vals`) or, when `offs`
// is given, the rule lengths offs[p + 1] - offs[p].
cudaError_t launch_vb_count(const u32* vals, const u64* offs, u64 n, u64* total, int sms, cudaStream_t st);
cudaError_t launch_vb_tile_bytes(const u32* vals, const u64* offs, u64 n, u32* tile_bytes, cudaStream_t st);
cudaError_t launch_vb_write(const u32* vals, const u64* offs, u64 n, const u64* tile_off, u8* out, bool pad,
                            cudaStream_t st);
cudaError_t launch_vb_tile_ends(const u8* in, u64 nb, u32* tile_cnt, cudaStream_t st);
cudaError_t launch_vb_dwrite(const u8* in, u64 nb, u64 n, u64 lo, u64 hi, const u64* cnt_off, u32* vals,
                             DevStatus* ds, cudaStream_t st);
u64 vb_encode_tiles(u64 n);
u64 vb_decode_tiles(u64 nb);

// Every column of a grammar in one launch per step: tile t of a launch
// belongs to the column c with cols[c].tile0 <= t < cols[c + 1].tile0; the
// entry after the last column holds the launch's tile count in tile0.
constexpr int kVbMaxCols = 2 * 64;
struct VbEncCol {
    const u32* vals;  // right-hand sides, or
    const u64* offs;  // rule offsets (the column holds the lengths)
    u64 n;            // values
    u64 tile0;        // first tile (of 2048 values)
    u8* dst;          // where the column's stream goes (set after the count)
};
struct VbDecCol {
    const u8* src;  // the column's stream
    u64 nb;         // its bytes
    u64 n;          // values it must hold
    u64 lo, hi;     // their range
    u32* out;
    u64 tile0;  // first tile (of 4096 bytes)
};
struct VbLevelOff {
    u64* rhs_off;  // g + 1 offsets to write
    u64 g, G;      // rules, symbols
    u64 gbase;     // the level's first length in the scanned array
};
cudaError_t launch_vb_tile_bytes_all(const VbEncCol* cols, u32 ncols, u64 tiles, u32* tile_bytes, u64* col_bytes,
                                     cudaStream_t st);
cudaError_t launch_vb_write_all(const VbEncCol* cols, u32 ncols, u64 tiles, const u64* tile_off, cudaStream_t st);
cudaError_t launch_vb_tile_ends_all(const VbDecCol* cols, u32 ncols, u64 tiles, u32* tile_cnt, cudaStream_t st);
cudaError_t launch_vb_dwrite_all(const VbDecCol* cols, u32 ncols, u64 tiles, const u64* cnt_off, DevStatus* ds,
                                 cudaStream_t st);
cudaError_t launch_vb_offsets_all(const VbLevelOff* lv, u32 nlv, u64 max_g, const u64* scan, const u64* total,
                                  DevStatus* ds, cudaStream_t st);

}  // namespace lcg
