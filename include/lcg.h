/*
 * lcg.h — C ABI of the GB300 library for stable locally consistent grammars.
 *
 * The library builds, merges and expands grammars of string collections with
 * the method of Diaz-Dominguez, "Efficient terabyte-scale text compression via
 * stable local consistency and parallel grammar processing" (arXiv 2411.12439):
 *
 *   BuildGram(T, H) = G      (Sec. 3.3; the operation is stated in Sec. 1)
 *   MergeGrams(G_a, G_b)     (Sec. 3.5-3.6)
 *   exp(C[j]) = T_j          (Sec. 2.2)
 *
 * and, on a finished grammar, the post-processing of Sec. 2.2 / Sec. 4
 * (run-length rules, then simplification: lcg_postprocess) and its VByte form
 * (Sec. 4, resource usage: lcg_export_vbyte / lcg_import_vbyte).
 *
 * Every step runs in hand-written CUDA kernels on one GPU (sm_103a).  There is
 * no CPU fallback: without a usable device every call returns LCG_EDEVICE.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * - Return value: LCG_OK (0) or a negative LCG_E* code.  The message of the
 *   last failure of a context is available from lcg_last_error().
 * - No C++ exception crosses this boundary.
 * - One context per host thread.  A context owns a CUDA stream on one device
 *   (the caller's stream when one is given).  All calls are blocking: when a
 *   call returns, its device work is complete.
 * - Grammars are owned by the library and live in the context's device
 *   memory until lcg_grammar_free().  Input and output buffers belong to the
 *   caller; the library never keeps a pointer to them after a call returns.
 * - Host pointers must be ordinary (pageable or pinned) host memory; device
 *   pointers must be device memory of the context's device.
 *
 * Grammar layout (Appendix A.1, with per-level ranks)
 * ----------------------------------------------------
 * Level 0 is the byte alphabet, with fingerprints F^0[s] = h^0(s), s = 0..255.
 * A level i >= 1 holds g^i rules.  Rule r (a 0-based rank in first-occurrence
 * order, see lcg_build) has right-hand side rhs[rhs_off[r] .. rhs_off[r+1]),
 * a sequence of level-(i-1) ranks (bytes at level 1), and fingerprint
 * F^i[r] = h^i(rhs) of Eq. fast_hash.  rhs_off has g^i+1 uint64 entries with
 * rhs_off[0] = 0, rhs is uint32 of length G^i = rhs_off[g^i], F^i is uint32.
 * The start rule S -> C[1..k] is stored as the pair (c_level[j], c_rank[j]):
 * the level and rank of the symbol that expands to string j.
 */
#ifndef LCG_H
#define LCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LCG_OK         0
#define LCG_EINVAL    -1  /* bad argument: k = 0, an empty string, bad level, ... */
#define LCG_ENOMEM    -2  /* device or host allocation failed */
#define LCG_ELEVELS   -3  /* the hash family has fewer functions than rounds needed */
#define LCG_EMISMATCH -4  /* grammars built with different hash families */
#define LCG_EOVERFLOW -5  /* a level would hold >= 2^32 rules, or a phrase >= 2^32 symbols */
#define LCG_ETIMEOUT  -6  /* a bounded device-side wait gave up */
#define LCG_EDEVICE   -7  /* CUDA error, or no usable device */
#define LCG_ETABLE    -8  /* phrase table could not be sized (after internal retries) */

typedef struct lcg_ctx lcg_ctx;
typedef struct lcg_grammar lcg_grammar;

/* The hash family H = {h^0, ..., h^{levels-1}} of Sec. 3.2.
 *
 * The paper draws, per level, a random prime p_i and a_i, b_i, c_i in [p_i]_+.
 * This library fixes p = 2^61 - 1 for every level and takes the random draws
 * as input: a[i], b[i], c[i] must lie in [1, 2^61 - 2].  m = 2^m_bits with
 * 1 <= m_bits <= 32 is the fingerprint range of every level.
 *   h^0(s)   = ((a_0 s + b_0) mod p) mod m                         (Sec. 2.4)
 *   h^i(Q)   = ((a_i (sum_{j=1..q} F^{i-1}[Q_j] c_i^{j-1}) + b_i) mod p) mod m
 *                                                      (Eq. lvl_hash / fast_hash)
 * The arrays are host memory and are copied by lcg_ctx_create.  A build needs
 * at least ceil(log2 n_max) + 1 functions (Sec. 3.2). */
typedef struct lcg_hash_family {
    uint32_t levels;
    uint32_t m_bits;
    const uint64_t* a;
    const uint64_t* b;
    const uint64_t* c;
} lcg_hash_family;

/* Per-round statistics of the last lcg_build / lcg_build_into of a context. */
typedef struct lcg_round_stats {
    uint64_t n;          /* |T^i|: symbols parsed in round i */
    uint64_t phrases;    /* phrases found in round i (= |T^{i+1}| before retiring) */
    uint64_t g;          /* new rules of level i */
    uint64_t G;          /* total length of their right-hand sides */
    uint64_t strings;    /* active strings entering round i */
    uint64_t table_cap;  /* phrase-table slots used for round i */
    uint32_t retries;    /* table regrowths in round i */
    uint32_t pad;
    double parse_ms;     /* device time of the round's k_parse launches (kernel timing on) */
    double round_ms;     /* device time of all the round's kernel launches (kernel timing
                            mode 1; with mode 2 only k_parse is timed) */
} lcg_round_stats;

typedef struct lcg_build_stats {
    uint32_t rounds;
    uint32_t async_rounds;      /* rounds enqueued without a host synchronisation,
                                   sized from the context's previous build */
    uint64_t kernel_launches;   /* kernels this library launched in the call */
    uint64_t input_bytes;
    uint32_t redone;            /* 1 when those planned rounds did not fit and the
                                   build was redone round by round */
    uint32_t graph;             /* 0: the rounds ran as launches; 1: they were captured
                                   into the context's CUDA graph and launched; 2: the
                                   graph captured for an earlier build was launched */
    lcg_round_stats round[64];
    double plan_slack;          /* the context's multiplier of planned buffer sizes after
                                   the call: it grows after a plan that did not fit and
                                   shrinks back towards 1 while plans fit */
} lcg_build_stats;

/* Device time of the kernels of the last call, per kernel kind (collected
 * only while kernel timing is enabled with lcg_set_kernel_timing). */
typedef struct lcg_kernel_time {
    char name[24];       /* kernel kind, e.g. "k_parse" */
    uint32_t launches;
    uint32_t pad;
    double ms;           /* summed CUDA-event time of its launches */
    double bytes;        /* algorithmic bytes of its launches (see the kernel's comment) */
} lcg_kernel_time;

/* Create a context on CUDA device `device` with hash family H.  `stream` is a
 * cudaStream_t to run on (NULL: the context creates its own).  Returns
 * LCG_EINVAL for a malformed family, LCG_EDEVICE when the device is not
 * usable. */
int lcg_ctx_create(int device, const lcg_hash_family* H, void* stream, lcg_ctx** out);
void lcg_ctx_destroy(lcg_ctx* ctx);
const char* lcg_last_error(const lcg_ctx* ctx);
/* Statistics of the last build call of this context (host struct filled). */
int lcg_last_build_stats(const lcg_ctx* ctx, lcg_build_stats* out);
/* Per-kernel CUDA-event timing in later calls: 0 off, 1 every kernel launch,
 * 2 only the parse launches (k_parse, the kernel with most device time, and
 * k_parse_small, the single-block parse of a short round; few
 * events, so the call's own time is barely changed).  Timed launches are
 * bracketed by two events on the context's stream; the sums are read with
 * lcg_last_kernel_times.  Other values give LCG_EINVAL. */
int lcg_set_kernel_timing(lcg_ctx* ctx, int enable);
/* Launch and sizing parameters of later builds (picked by an autotuner, e.g.
 * paper_2411_12439_gb300/autotune.py; the results do not depend on them):
 *   table_load          phrase-table slots per expected new rule is 1 / table_load
 *                       (0.3 .. 0.78; a table past 0.8 is regrown and the round rerun);
 *   parse_blocks_per_sm resident k_parse blocks per SM, 0 = as many as fit;
 *   miss_flush          byte rounds: queued cache misses that trigger a lookup pass
 *                       (32 .. 256; at most 128 take effect with 4096-position tiles);
 *   table_slots_max     0, or at most this many slots (>= 1024) in the first phrase
 *                       table of every round: a table too small for the round fills
 *                       past its load limit, is regrown (x4) and the parse rerun, so
 *                       the regrowth path can be exercised; results are unchanged;
 *   tile_stripes        rounds >= 2 take their parse tiles in this many interleaved
 *                       stripes of the sequence (1 .. 16; 1 = in order), so that
 *                       strings that are near-copies of one another at the same
 *                       offsets are parsed side by side;
 *   parse_tile          positions per parse tile: 1024, 2048 or 4096.  A block of
 *                       k_parse stages, lists and looks up one tile at a time (fewer
 *                       barriers per phrase with larger tiles, more blocks' worth of
 *                       tiles in flight with smaller ones);
 *   parse_tile_min      a round's tile is halved (down to 1024 positions) while the
 *                       round would have fewer than this many tiles per SM (0 .. 1024;
 *                       0 keeps every round at parse_tile).
 * Defaults: 0.35, 0, 64, 0, 1, 4096, 16.  Out-of-range values give LCG_EINVAL. */
typedef struct lcg_tuning {
    double table_load;
    uint32_t parse_blocks_per_sm;
    uint32_t miss_flush;
    uint32_t table_slots_max;
    uint32_t tile_stripes;
    uint32_t parse_tile;
    uint32_t parse_tile_min;
} lcg_tuning;
int lcg_set_tuning(lcg_ctx* ctx, const lcg_tuning* t);
/* Run later lcg_build calls whose rounds are planned without host
 * synchronisation as one CUDA graph (1) or as launches (0, the default).  The
 * first build of a shape (device input buffer, string lengths, plan) captures
 * the graph; later builds of that shape launch it, provided the grammar of the
 * previous launch has been freed (the graph writes the grammar into its own
 * allocations, at the same addresses every time); otherwise, and for
 * collections with strings of length one, the build runs as launches.  Input
 * in host memory is first copied into an upload buffer that the context keeps
 * (grown when needed), so that its builds can launch the graph too.  Results
 * do not depend on it. */
int lcg_set_graph(lcg_ctx* ctx, int enable);
int lcg_get_tuning(const lcg_ctx* ctx, lcg_tuning* t);

/* Copy up to `cap` entries of the per-kind kernel times of the last call into
 * `out` (host) and their number into *count. */
int lcg_last_kernel_times(const lcg_ctx* ctx, lcg_kernel_time* out, uint32_t cap, uint32_t* count);

/* One timed kernel launch of the last call (kernel timing on). */
typedef struct lcg_kernel_launch {
    char name[24];       /* kernel kind, e.g. "k_parse" */
    uint32_t round;      /* BuildGram round of a build's launch (1 = bytes), 0 for others */
    uint32_t pad;
    double ms;           /* CUDA-event time of the launch */
    double bytes;        /* algorithmic bytes of the launch */
} lcg_kernel_launch;
/* Copy up to `cap` of the last call's timed launches, in launch order, into
 * `out` (host) and their number into *count. */
int lcg_last_kernel_launches(const lcg_ctx* ctx, lcg_kernel_launch* out, uint32_t cap, uint32_t* count);

/* Self-test of the bounded device waits (no counterpart in the paper; the
 * failure detection of the library).  Runs the library's single-pass scan on
 * a small array with its tile counter read one ahead, so that the first tile
 * waits for a predecessor that never publishes.  The wait gives up after its
 * iteration limit (about a second), the kernel records the timeout in the
 * context's device status and returns, and the call returns LCG_ETIMEOUT.
 * Nothing faults, traps or hangs, and later calls on the context work as
 * before (look-back slots carry a launch epoch).  Any other return value means
 * the bounded wait is broken. */
int lcg_selftest_wait_timeout(lcg_ctx* ctx);

/* BuildGram(T, H) (Sec. 3.3).
 * data: the k strings concatenated (uint8), `data_on_device` = 1 when it is a
 *       device pointer, 0 when it is host memory (copied in by the call).
 * offsets: HOST array of k+1 uint64; string j is data[offsets[j] .. offsets[j+1]).
 * Every string must be non-empty (LCG_EINVAL otherwise).
 * Rounds i = 1, 2, ... break every active string at the LMS positions of
 * RandLMSPar (Eq. rand_types), give each distinct phrase of the round a rank
 * of level i in order of first occurrence over the concatenated active strings
 * (string index, then position), and replace the phrases by their ranks.  A
 * string whose sequence has length one after round i is done: C[j] = (i, rank).
 * A string of length one on input has C[j] = (0, byte).
 * On success *out is a new device-resident grammar. */
int lcg_build(lcg_ctx* ctx, const uint8_t* data, const uint64_t* offsets, uint32_t k,
              int data_on_device, lcg_grammar** out);

/* The parse of Appendix A.2 against a resident grammar: strings T are parsed
 * with the same rounds as lcg_build, a phrase that is already a rule of the
 * resident grammar keeps its rank, and new phrases are appended after the
 * resident rules of their level in first-occurrence order.  The result is
 * identical to lcg_merge(resident, lcg_build(T)).  `resident` is modified in
 * place; its C grows by k entries. */
int lcg_build_into(lcg_ctx* ctx, lcg_grammar* resident, const uint8_t* data, const uint64_t* offsets,
                   uint32_t k, int data_on_device);

/* MergeGrams(G_a, G_b) (Sec. 3.6): `a` absorbs `b` (b is left unchanged).
 * Level by level, every rule of b whose right-hand side (rewritten into a's
 * ranks of the level below) is a rule of a maps to that rule; the others are
 * appended to a in b's rank order.  C_a becomes C_a . C_b.  Grammars built
 * with different hash families give LCG_EMISMATCH. */
int lcg_merge(lcg_ctx* ctx, lcg_grammar* a, const lcg_grammar* b);

/* exp(C[j]) (Sec. 2.2).  Writes min(cap, |T_j|) bytes to `out` (device memory
 * when out_on_device = 1, else host) and the full length to *out_len; returns
 * LCG_EINVAL when cap < |T_j| (nothing is written then) or j >= k. */
int lcg_decompress(lcg_ctx* ctx, const lcg_grammar* G, uint32_t j, uint8_t* out, uint64_t cap,
                   uint64_t* out_len, int out_on_device);

/* exp(C[j]) like lcg_decompress, but without allocating any device memory.
 * This entry point has no counterpart in the paper; it is a library service
 * for callers that cannot allocate device memory when they expand a string:
 * code running inside an allocator's or a memory-pressure callback (it cannot
 * call back into the allocator), and services that reserve their device
 * memory up front and keep no room for transient buffers.  Its scratch is a
 * static device array of about 20 MiB, which every GPU that loads the library
 * keeps until the process exits.  The context and the grammar must already
 * exist.
 * out_dev: DEVICE buffer of `cap` bytes; on success *out_len receives |T_j|.
 * Limits and errors: a string longer than 1048576 bytes is rejected with
 * LCG_EOVERFLOW, and *out_len then holds only a lower bound of its length (the
 * expansion stops at the first level past the limit; use lcg_decompress);
 * cap < |T_j| gives LCG_EINVAL with *out_len = |T_j|; j >= k gives LCG_EINVAL.
 * The first call on a device takes the scratch's device address
 * (cudaGetSymbolAddress, once per device): make that first call before any
 * stream capture.  All calls share the scratch and it keeps the last call's
 * contents: calls whose device work overlaps (other threads, other contexts or
 * streams) race and must be serialised by the caller.  The call blocks: it
 * synchronises the context's stream at every level to read the size of the
 * next level's expansion back from the device. */
int lcg_decompress_static(lcg_ctx* ctx, const lcg_grammar* G, uint32_t j, uint8_t* out_dev, uint64_t cap,
                          uint64_t* out_len);

/* Shape of a grammar: number of strings k and of levels >= 1. */
int lcg_grammar_shape(const lcg_grammar* G, uint32_t* k, uint32_t* nlevels);
/* Sizes of level i >= 1: g^i rules and G^i right-hand-side symbols. */
int lcg_level_size(const lcg_grammar* G, uint32_t level, uint64_t* g, uint64_t* Gsz);
/* Copy level i >= 1 to host buffers of g+1, G and g entries (any may be NULL). */
int lcg_export_level(lcg_ctx* ctx, const lcg_grammar* G, uint32_t level, uint64_t* rhs_off,
                     uint32_t* rhs, uint32_t* F);
/* Copy F^0 (256 entries) and C (k entries each) to host buffers. */
int lcg_export_start(lcg_ctx* ctx, const lcg_grammar* G, uint32_t* F0, uint32_t* c_level, uint32_t* c_rank);

/* A device grammar from host arrays in the layout of lcg_export_level and
 * lcg_export_start: the way a grammar built by another process or GPU enters
 * this context before MergeGrams (Sec. 3.6; the per-GPU grammars of a sharded
 * collection are merged this way).
 * k strings and nlevels levels.  For level i = 1..nlevels (array index i-1):
 *   g[i-1]        rules;
 *   rhs_off[i-1]  g+1 uint64 offsets, starting at 0 and strictly increasing;
 *   rhs[i-1]      rhs_off[i-1][g] uint32 symbols, each a rank of level i-1
 *                 (a byte value at level 1);
 *   F[i-1]        g uint32 fingerprints F^i.
 * c_level, c_rank: k entries; (level, rank) of exp(T_j) as in C (Sec. 3.3).
 * F^0 is not passed: it comes from the context's hash family.
 * All pointers are HOST pointers, read during the call and not retained; the
 * new grammar (*out) belongs to the library.
 * Errors: malformed arrays (offsets, a symbol or C entry naming a missing rule)
 * give LCG_EINVAL; nlevels not below the family's length LCG_ELEVELS; every
 * F^i[r] is recomputed on the device from the right-hand side with Eq. fast_hash
 * and a difference (a grammar of another hash family) gives LCG_EMISMATCH.
 * The call is blocking. */
int lcg_import(lcg_ctx* ctx, uint32_t k, uint32_t nlevels, const uint64_t* g, const uint64_t* const* rhs_off,
               const uint32_t* const* rhs, const uint32_t* const* F, const uint32_t* c_level, const uint32_t* c_rank,
               lcg_grammar** out);
/* Roots of strings j0 .. j0+count-1 of G: C[j] = (level[x], rank[x]) and the
 * fingerprint fp[x] = F^level[rank] of exp(T_j) (F^0 for a string of length
 * one).  The fingerprint depends on the string's content only (Eq. fast_hash):
 * it is the same whichever strings the grammar holds besides T_j.  Outputs are
 * HOST arrays of `count` entries.  LCG_EINVAL when j0 + count > k.  Blocking. */
int lcg_string_roots(lcg_ctx* ctx, const lcg_grammar* G, uint32_t j0, uint32_t count, uint32_t* level,
                     uint32_t* rank, uint32_t* fp);

/* The packed form of a grammar: one buffer, for storage and for sending a
 * grammar to another process (the merge tree of a sharded collection).
 * Layout (little-endian; every array starts at a multiple of 8 bytes, u32
 * arrays are zero-padded to a multiple of 8 bytes):
 *   u64 magic 0x4C434753, u64 k, u64 nlevels, then per level (u64 g, u64 G);
 *   per level: u64 rhs_off[g+1], u32 rhs[G], u32 F[g];
 *   u32 c_level[k], u32 c_rank[k], u32 F0[256].
 * lcg_packed_size gives its size in bytes. */
int lcg_packed_size(const lcg_grammar* G, uint64_t* bytes);
/* Write G's packed form into the HOST buffer `out` (8-byte aligned, `cap`
 * bytes, at least lcg_packed_size); page-locked memory lets the copies run at
 * link speed.  Blocking.  LCG_EINVAL when the buffer is too small or
 * misaligned. */
int lcg_export_packed(lcg_ctx* ctx, const lcg_grammar* G, void* out, uint64_t cap);
/* A device grammar from a packed HOST buffer of `size` bytes (8-byte
 * aligned), with the checks of lcg_import; an F0 other than this context's
 * gives LCG_EMISMATCH, a malformed buffer LCG_EINVAL.  Blocking. */
int lcg_import_packed(lcg_ctx* ctx, const void* buf, uint64_t size, lcg_grammar** out);

/* ---- VByte (Sec. 4, resource usage: grammar symbols stored with VBytes
 * instead of 32-bit cells) ----
 *
 * A value (< 2^32) is cut into groups of 7 bits, least significant group
 * first, one group per byte; the high bit of a byte is set when another byte
 * of the same value follows (the LEB128 / varint layout).  A value takes
 * 1 to 5 bytes.
 *
 * lcg_vbyte_encode: the VByte stream of the n values of the DEVICE array
 * `in`, written to the DEVICE buffer `out` of `cap` bytes; *out_bytes gets the
 * stream's length (also when `cap` is too small, which gives LCG_EINVAL and
 * writes nothing).  Blocking.
 * lcg_vbyte_decode: exactly `n` values from the `nbytes`-byte DEVICE stream
 * `in` into the DEVICE array `out`.  A stream that ends inside a value, holds a
 * value of more than 32 bits or 5 bytes, or holds another number of values
 * gives LCG_EINVAL (the output is then undefined).  Blocking. */
int lcg_vbyte_encode(lcg_ctx* ctx, const uint32_t* in, uint64_t n, uint8_t* out, uint64_t cap, uint64_t* out_bytes);
int lcg_vbyte_decode(lcg_ctx* ctx, const uint8_t* in, uint64_t nbytes, uint32_t* out, uint64_t n);

/* The VByte form of a grammar: the packed form with every level's rule
 * lengths and right-hand sides in VByte.
 * Layout (little-endian; every section starts at a multiple of 8 bytes and
 * is zero-padded):
 *   u64 magic 0x4C434756, u64 k, u64 nlevels,
 *   per level: u64 g, u64 G, u64 bytes of the lengths, u64 bytes of the symbols;
 *   per level: VByte of |rhs(X)| for the g rules in rank order,
 *              VByte of the G right-hand-side symbols, u32 F[g];
 *   u32 c_level[k], u32 c_rank[k], u32 F0[256].
 * lcg_vbyte_size: its size in bytes (reads the grammar on the device;
 * blocking).
 * lcg_export_vbyte: writes it into `out` (`cap` bytes, 8-byte aligned; a
 * DEVICE buffer when out_on_device, else HOST memory, page-locked for speed);
 * *bytes (optional) gets the size.  LCG_EINVAL when the buffer is too small or
 * misaligned.  Blocking.
 * lcg_import_vbyte: a device grammar from a VByte form of `size` bytes (a
 * DEVICE buffer when buf_on_device, else HOST memory; 8-byte aligned), with
 * the checks of lcg_import: a malformed buffer or stream gives LCG_EINVAL,
 * fingerprints or F0 of another hash family LCG_EMISMATCH.  Blocking. */
int lcg_vbyte_size(lcg_ctx* ctx, const lcg_grammar* G, uint64_t* bytes);
int lcg_export_vbyte(lcg_ctx* ctx, const lcg_grammar* G, void* out, uint64_t cap, int out_on_device,
                     uint64_t* bytes);
int lcg_import_vbyte(lcg_ctx* ctx, const void* buf, uint64_t size, int buf_on_device, lcg_grammar** out);
/* Release a grammar (NULL is ignored).  While the context that created it
 * exists, the device memory returns to the pool in the order of that
 * context's stream, so later calls of the context reuse it at no cost; after
 * lcg_ctx_destroy it is freed at once.  A grammar must not be freed while a
 * call that uses it runs on another host thread. */
void lcg_grammar_free(lcg_grammar* G);

/* ---- post-processing: run-length rules (RL), then simplification (Simp) ----
 *
 * Sec. 2.2 (post-processing) and Sec. 4 (the tool runs RL, then Simp, on the
 * output of BuildGram).  RL: every maximal run Y^l (l >= 2) of one symbol in
 * the right-hand side of one rule of level i becomes a reference to a
 * run-length rule (Y, l) of level i; the distinct pairs of a level are
 * numbered by first occurrence (rule rank, then position).  Runs never cross
 * rule boundaries and the roots C are left as they are.  Simp: a rule of level
 * i that occurs exactly once in the right-hand sides of level i+1, and is
 * neither a string's root nor the base of a run-length rule, is removed and
 * its occurrence replaced by its right-hand side (recursively); run-length
 * rules are never removed.
 *
 * The result is one grammar over global ids: 0..255 are the bytes; then, level
 * by level, the surviving rules in rank order followed by the level's
 * run-length rules get the ids 256, 257, ...  Rule x - 256 has kind 0 (its
 * right-hand side is a list of ids) or kind 1 (a run-length rule stored as the
 * two entries [base id, run length]); c[j] is the id of string j's root.  The
 * grammar's size is the total right-hand-side length.
 *
 * lcg_postprocess reads G (unchanged; it may still be used, merged or freed)
 * and returns a new device-resident object owned by the caller, freed with
 * lcg_pp_free.  Errors: LCG_EINVAL (null arguments, another device, more than
 * 64 levels), LCG_EOVERFLOW (2^32 output ids or more), LCG_ENOMEM, LCG_EDEVICE.
 * lcg_pp_export copies the arrays to host buffers of sizes taken from
 * lcg_pp_stats_of (kind: rules bytes; rhs_off: rules + 1 uint64; rhs: size
 * uint32; c: strings uint32) and synchronises the device. */
typedef struct lcg_pp lcg_pp;
typedef struct lcg_pp_stats {
    uint64_t size_before;  /* total right-hand-side length of the level grammar */
    uint64_t size_rl;      /* after RL (a run-length rule counts two) */
    uint64_t size;         /* after Simp: the result's size */
    uint64_t rl_rules;     /* run-length rules created */
    uint64_t removed;      /* rules removed by Simp */
    uint64_t rules;        /* rules of the result (ids 256 .. 256 + rules - 1) */
    uint64_t strings;      /* roots c[0 .. strings - 1] */
} lcg_pp_stats;
int lcg_postprocess(lcg_ctx* ctx, const lcg_grammar* G, lcg_pp** out);
int lcg_pp_stats_of(const lcg_pp* pp, lcg_pp_stats* out);
int lcg_pp_export(const lcg_pp* pp, uint8_t* kind, uint64_t* rhs_off, uint32_t* rhs, uint32_t* c);
void lcg_pp_free(lcg_pp* pp);

#ifdef __cplusplus
}
#endif

#endif /* LCG_H */
