// C ABI of the library (include/lcg.h): contexts, the BuildGram round driver
// (rounds enqueued without host synchronisation, and their CUDA graph),
// MergeGrams, expansion, export / import and post-processing.  Host code only
// orchestrates: every step of the method runs in the kernels of parse.cu,
// grammar.cu and post.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lcg.h"
#include "lcg_internal.h"

using namespace lcg;

// --------------------------------------------------------------------------
// objects
// --------------------------------------------------------------------------

namespace {

struct Level {
    u64 g = 0, G = 0;          // rules and right-hand-side symbols
    u64 cap_g = 0, cap_G = 0;  // allocated capacity
    u64* rhs_off = nullptr;    // cap_g + 1 entries
    u32* rhs = nullptr;
    u32* F = nullptr;
    void* rtab = nullptr;      // table over the rules (for parses against this grammar and merges)
    u64 rcap = 0;
    bool rvalid = false;
};

}  // namespace

struct lcg_grammar {
    int device = 0;
    lcg_ctx* owner = nullptr;  // the context that created it, while that context lives
    u64 tag = 0;
    u32* F0 = nullptr;  // 256 fingerprints of bytes (device)
    std::vector<Level> lv;
    u32 k = 0, cap_k = 0;
    u32* c_level = nullptr;
    u32* c_rank = nullptr;
};

namespace {
struct GraphBuild;
}

struct lcg_ctx {
    int device = 0;
    int sms = 1;                         // SMs of the device
    bool use_graph = false;              // builds may run as a captured CUDA graph
    GraphBuild* graph = nullptr;         // the graph of the last shape
    cudaStream_t st = nullptr;
    std::vector<lcg_grammar*> live;  // grammars created here and not yet freed
    double plan_slack = 1.0;         // multiplier of the planned buffer sizes (adaptive)
    // table load, k_parse blocks per SM, miss flush, slots cap, stripes, parse tile
    lcg_tuning tuning{0.35, 0, 64, 0, 1, 4096, 16};
    bool own_stream = false;
    std::vector<u64> a, b, c;
    u32 levels = 0, m_bits = 32;
    u64 mmask = 0xffffffffull;
    u64 tag = 0;
    std::string err;
    // persistent device scratch
    DevStatus* ds = nullptr;
    RoundCounts* rc = nullptr;
    u64* ctr = nullptr;     // tile counter of single-pass kernels (never reset)
    u64 ctr_val = 0;        // its value after all launched tiles ran
    u64 epoch = 0;          // look-back epoch, one per launch
    u64* scratch = nullptr; // small device scalars: [0] phrases, [1..2] totals
    void* lb1 = nullptr;
    u64 lb1_tiles = 0;
    void* heads = nullptr;  // k_breaks' look-ahead words (its own: epoch-tagged, nothing else writes them)
    u64 heads_steps = 0;
    void* lb2 = nullptr;
    u64 lb2_tiles = 0;
    double ratio_hint[64] = {0};  // new rules per phrase, per level (decaying maximum over builds)
    double p_hint[64] = {0};      // phrases per symbol, per level (decaying maximum)
    double glen_hint[64] = {0};   // symbols per new rule, per level (decaying maximum)
    u32 hint_rounds = 0;          // rounds of the last build (0: none yet)
    // per-round device status, counts and totals (rounds enqueued without syncs)
    DevStatus* ds_arr = nullptr;
    RoundCounts* rc_arr = nullptr;
    u64* tot_arr = nullptr;
    lcg_build_stats stats{};
    u64 launches = 0;
    // per-kernel CUDA-event timing (optional)
    int ktime = 0;  // 0 off, 1 every launch, 2 parse launches only
    bool capturing = false;              // the stream is being captured into a graph
    unsigned char* upload = nullptr;     // host input of graph builds, at a fixed address
    u64 upload_cap = 0;
    struct KRec {
        const char* name;
        cudaEvent_t a, b;
        double bytes;
        u32 round;  // BuildGram round of a parse launch, else 0
        bool graph;  // the events belong to a captured graph
    };
    std::vector<KRec> krecs;
    std::vector<cudaEvent_t> evpool;
    std::vector<lcg_kernel_time> ktimes;
    std::vector<lcg_kernel_launch> klaunches;
};

namespace {

constexpr u64 kMaxRank = 0x7fffffffull;  // ranks are tagged with one bit in the phrase slots
constexpr u32 kMaxRounds = 63;

struct Fail {
    int code;
};

void fail_if(lcg_ctx* ctx, bool cond, int code, const std::string& msg) {
    if (cond) {
        ctx->err = msg;
        throw Fail{code};
    }
}

void ck(lcg_ctx* ctx, cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
        throw Fail{e == cudaErrorMemoryAllocation ? LCG_ENOMEM : LCG_EDEVICE};
    }
}

template <typename T>
T* dalloc(lcg_ctx* ctx, u64 count) {
    void* p = nullptr;
    if (count == 0) count = 1;
    ck(ctx, cudaMallocAsync(&p, count * sizeof(T), ctx->st), "cudaMallocAsync");
    return (T*)p;
}

void dfree(lcg_ctx* ctx, void* p) {
    if (p) cudaFreeAsync(p, ctx->st);
}

void sync(lcg_ctx* ctx) { ck(ctx, cudaStreamSynchronize(ctx->st), "stream synchronize"); }

// ---- per-kernel timing: events around each launch when enabled -----------

cudaEvent_t kt_event(lcg_ctx* ctx) {
    if (!ctx->evpool.empty()) {
        cudaEvent_t e = ctx->evpool.back();
        ctx->evpool.pop_back();
        return e;
    }
    cudaEvent_t e;
    ck(ctx, cudaEventCreate(&e), "cudaEventCreate");
    return e;
}

// Under stream capture a plain record only marks a dependency; an external
// record becomes an event node that the graph records at every launch.
cudaError_t record_event(lcg_ctx* ctx, cudaEvent_t e) {
    return ctx->capturing ? cudaEventRecordWithFlags(e, ctx->st, cudaEventRecordExternal) : cudaEventRecord(e, ctx->st);
}

void kt_reset(lcg_ctx* ctx) {
    for (auto& r : ctx->krecs) {
        if (r.graph) continue;  // recorded by a graph's event nodes: the graph owns them
        ctx->evpool.push_back(r.a);
        ctx->evpool.push_back(r.b);
    }
    ctx->krecs.clear();
    ctx->ktimes.clear();
    ctx->klaunches.clear();
}

// Record the start of a launch of kernel `name` that moves `bytes` algorithmic
// bytes; returns a handle for kt_end (or -1 when timing is off).
int kt_begin(lcg_ctx* ctx, const char* name, double bytes, u32 round = 0) {
    // mode 2: the parse launches only (k_parse, and k_parse_small of short rounds)
    if (ctx->ktime == 0 || (ctx->ktime == 2 && std::strncmp(name, "k_parse", 7) != 0)) return -1;
    lcg_ctx::KRec r{name, kt_event(ctx), kt_event(ctx), bytes, round, false};
    ck(ctx, record_event(ctx, r.a), "cudaEventRecord");
    ctx->krecs.push_back(r);
    return (int)ctx->krecs.size() - 1;
}

void kt_end(lcg_ctx* ctx, int h) {
    if (h >= 0) ck(ctx, record_event(ctx, ctx->krecs[h].b), "cudaEventRecord");
}

// After the call's last synchronisation: sum the times per kernel kind.
void kt_collect(lcg_ctx* ctx) {
    ctx->ktimes.clear();
    ctx->klaunches.clear();
    for (auto& r : ctx->krecs) {
        float ms = 0.f;
        ck(ctx, cudaEventElapsedTime(&ms, r.a, r.b), "cudaEventElapsedTime");
        lcg_kernel_launch kl{};
        std::strncpy(kl.name, r.name, sizeof(kl.name) - 1);
        kl.round = r.round;
        kl.ms = ms;
        kl.bytes = r.bytes;
        ctx->klaunches.push_back(kl);
        lcg_kernel_time* t = nullptr;
        for (auto& x : ctx->ktimes)
            if (std::strncmp(x.name, r.name, sizeof(x.name)) == 0) t = &x;
        if (!t) {
            lcg_kernel_time z{};
            std::strncpy(z.name, r.name, sizeof(z.name) - 1);
            ctx->ktimes.push_back(z);
            t = &ctx->ktimes.back();
        }
        t->launches++;
        t->ms += ms;
        t->bytes += r.bytes;
        if (r.round >= 1 && r.round <= 64) {
            lcg_round_stats& rs = ctx->stats.round[r.round - 1];
            rs.round_ms += ms;
            if (std::strcmp(r.name, "k_parse") == 0) rs.parse_ms += ms;
        }
    }
}

void check_device_status(lcg_ctx* ctx, const DevStatus& h) {
    switch (h.error) {
        case kErrNone: return;
        case kErrTimeout: fail_if(ctx, true, LCG_ETIMEOUT, "a bounded device wait gave up"); break;
        case kErrTableFull: fail_if(ctx, true, LCG_ETABLE, "phrase table full"); break;
        case kErrPhraseLong: fail_if(ctx, true, LCG_EOVERFLOW, "phrase of 2^32 symbols or more"); break;
        case kErrMismatch: fail_if(ctx, true, LCG_EMISMATCH, "equal rules with different fingerprints"); break;
        case kErrFormat: fail_if(ctx, true, LCG_EINVAL, "malformed VByte stream"); break;
        default: fail_if(ctx, true, LCG_EDEVICE, "device error " + std::to_string(h.error));
    }
}

// A call starts with a clear status: an error of an earlier call does not
// carry over.
void reset_status(lcg_ctx* ctx) {
    ck(ctx, cudaMemsetAsync(ctx->ds, 0, sizeof(DevStatus), ctx->st), "reset status");
}

DevStatus read_status(lcg_ctx* ctx) {
    DevStatus h;
    ck(ctx, cudaMemcpyAsync(&h, ctx->ds, sizeof(h), cudaMemcpyDeviceToHost, ctx->st), "read status");
    sync(ctx);
    return h;
}

LevelHash level_hash(const lcg_ctx* ctx, u32 i) {
    LevelHash h;
    h.a = ctx->a[i];
    h.b = ctx->b[i];
    h.c = ctx->c[i];
    h.mmask = ctx->mmask;
    return h;
}

// The planned rounds did not fit (or a graph capture had to be abandoned):
// the build is redone round by round.
struct Retry {};

void destroy_graph(lcg_ctx* ctx);

// NVTX range for profilers (a no-op when no tool is attached): calls, rounds.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    Range(const char* what, u32 i) {
        char b[48];
        std::snprintf(b, sizeof(b), "%s %u", what, i);
        nvtxRangePushA(b);
    }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

void ensure_lb(lcg_ctx* ctx, void** lb, u64* have, u64 tiles, size_t bytes) {
    if (tiles <= *have) return;
    u64 want = std::max<u64>(tiles, *have * 2);
    size_t nb = bytes / (tiles ? tiles : 1) * want;
    // a graph being captured has its buffers sized beforehand; should one
    // not fit, the capture is abandoned and the build runs round by round
    if (ctx->capturing) throw Retry{};
    // a captured graph uses the current look-back buffers: it goes with them
    if (*lb && ctx->graph) destroy_graph(ctx);
    if (*lb) dfree(ctx, *lb);
    void* p = nullptr;
    ck(ctx, cudaMallocAsync(&p, nb, ctx->st), "cudaMallocAsync lb");
    ck(ctx, cudaMemsetAsync(p, 0, nb, ctx->st), "memset lb");
    *lb = p;
    *have = want;
}

// grow a level's arrays to hold `need_g` rules and `need_G` symbols
void grow_level(lcg_ctx* ctx, Level& L, u64 need_g, u64 need_G) {
    if (need_g > L.cap_g || L.rhs_off == nullptr) {
        u64 cap = std::max<u64>(need_g, std::max<u64>(L.cap_g * 2, 256));
        u64* ro = dalloc<u64>(ctx, cap + 1);
        u32* F = dalloc<u32>(ctx, cap);
        if (L.rhs_off) {
            ck(ctx, cudaMemcpyAsync(ro, L.rhs_off, (L.g + 1) * sizeof(u64), cudaMemcpyDeviceToDevice, ctx->st), "copy");
            ck(ctx, cudaMemcpyAsync(F, L.F, L.g * sizeof(u32), cudaMemcpyDeviceToDevice, ctx->st), "copy");
            dfree(ctx, L.rhs_off);
            dfree(ctx, L.F);
        } else {
            ck(ctx, cudaMemsetAsync(ro, 0, sizeof(u64), ctx->st), "memset");
        }
        L.rhs_off = ro;
        L.F = F;
        L.cap_g = cap;
    }
    if (need_G > L.cap_G || L.rhs == nullptr) {
        u64 cap = std::max<u64>(need_G, std::max<u64>(L.cap_G * 2, 1024));
        u32* r = dalloc<u32>(ctx, cap);
        if (L.rhs) {
            ck(ctx, cudaMemcpyAsync(r, L.rhs, L.G * sizeof(u32), cudaMemcpyDeviceToDevice, ctx->st), "copy");
            dfree(ctx, L.rhs);
        }
        L.rhs = r;
        L.cap_G = cap;
    }
}

const u32* fprev_of(const lcg_grammar* G, u32 i) { return i == 1 ? G->F0 : G->lv[i - 2].F; }

// (Re)build the table over the rules of level i so that it can take
// `need_g` rules at load <= 1/2.
void ensure_resident(lcg_ctx* ctx, lcg_grammar* G, u32 i, u64 need_g) {
    Level& L = G->lv[i - 1];
    if (L.rvalid && L.rcap >= 2 * need_g) return;
    const u64 cap = std::max<u64>(1024, 3 * need_g);
    dfree(ctx, L.rtab);
    L.rtab = dalloc<unsigned char>(ctx, cap * slot_bytes());
    L.rcap = cap;
    ck(ctx, cudaMemsetAsync(L.rtab, 0xFF, cap * slot_bytes(), ctx->st), "memset table");
    ck(ctx, launch_resident_build(L.rhs, L.rhs_off, 0, L.g, i == 1, fprev_of(G, i), level_hash(ctx, i), L.rtab,
                                  cap, ctx->ds, ctx->st),
       "resident build");
    ctx->launches++;
    L.rvalid = true;
}

void grow_c(lcg_ctx* ctx, lcg_grammar* G, u32 need) {
    if (need <= G->cap_k && G->c_level) return;
    u32 cap = std::max<u32>(need, std::max<u32>(G->cap_k * 2, 16));
    u32* cl = dalloc<u32>(ctx, cap);
    u32* cr = dalloc<u32>(ctx, cap);
    if (G->c_level) {
        ck(ctx, cudaMemcpyAsync(cl, G->c_level, G->k * sizeof(u32), cudaMemcpyDeviceToDevice, ctx->st), "copy");
        ck(ctx, cudaMemcpyAsync(cr, G->c_rank, G->k * sizeof(u32), cudaMemcpyDeviceToDevice, ctx->st), "copy");
        dfree(ctx, G->c_level);
        dfree(ctx, G->c_rank);
    }
    G->c_level = cl;
    G->c_rank = cr;
    G->cap_k = cap;
}

// A grammar with no strings yet: F^0 on the device.  `registered`: the
// context tracks it (every grammar handed to a caller).
lcg_grammar* new_grammar(lcg_ctx* ctx, bool registered = true) {
    lcg_grammar* G = new lcg_grammar();
    G->device = ctx->device;
    G->tag = ctx->tag;
    if (registered) {
        G->owner = ctx;
        ctx->live.push_back(G);
    }
    G->F0 = dalloc<u32>(ctx, 256);
    ck(ctx, launch_h0(level_hash(ctx, 0), G->F0, ctx->st), "h0");
    ctx->launches++;
    return G;
}

void graph_grammar_freed(lcg_ctx* ctx, const lcg_grammar* G);

// Release a grammar.  While its context lives, the memory goes back to the
// pool in the order of that context's stream (later calls reuse it without a
// device synchronisation); otherwise it is freed at once.
void free_grammar_now(lcg_grammar* G) {
    if (!G) return;
    cudaSetDevice(G->device);
    cudaStream_t st = nullptr;
    if (G->owner) {
        auto& v = G->owner->live;
        v.erase(std::remove(v.begin(), v.end(), G), v.end());
        st = G->owner->st;
        graph_grammar_freed(G->owner, G);
    }
    auto release = [&](void* p) {
        if (!p) return;
        if (st) cudaFreeAsync(p, st); else cudaFree(p);
    };
    release(G->F0);
    for (Level& L : G->lv) {
        release(L.rhs_off);
        release(L.rhs);
        release(L.F);
        release(L.rtab);
    }
    release(G->c_level);
    release(G->c_rank);
    delete G;
}

// --------------------------------------------------------------------------
// BuildGram round driver
// --------------------------------------------------------------------------

// Per-round ratios that size the next build's buffers: the largest seen,
// decaying by 10 % per build, so that a context that sees collections of
// changing make-up (a serving loop) keeps plans that fit.
void record_hints(lcg_ctx* ctx, u32 i, u64 n, u64 P, u64 g, u64 G) {
    if (i >= 64) return;
    // the largest ratio seen, fading by 2 % per build: a context fed collections
    // of changing make-up (a serving lane) keeps plans that fit its larger ones
    auto keep = [](double old, double x) { return std::max(x, 0.98 * old); };
    ctx->ratio_hint[i] = keep(ctx->ratio_hint[i], P ? (double)g / (double)P : 0.0);
    ctx->p_hint[i] = keep(ctx->p_hint[i], n ? (double)P / (double)n : 0.0);
    ctx->glen_hint[i] = keep(ctx->glen_hint[i], g ? (double)G / (double)g : 2.0);
}

// The sequence a round reads: T^i, its fingerprints (rounds >= 2) and the
// offsets and ids of its active strings.
struct RoundInput {
    const void* S;
    void* S_owned;
    const u32* Sf;
    int symb;
    u64 n;          // |T^i| (host value when known)
    u32 kk;         // active strings (host value when known)
    u64* soff;
    u32* sid;
    const u64* d_n;  // device values, for rounds enqueued without a sync
    const u64* d_k;
    bool own_offsets = true;  // soff / sid are this build's to free
};


void free_round_input(lcg_ctx* ctx, RoundInput& in) {
    if (in.own_offsets) {
        dfree(ctx, in.soff);
        dfree(ctx, in.sid);
    }
    if (in.S_owned) dfree(ctx, in.S_owned);
    if (in.Sf) dfree(ctx, (void*)in.Sf);
    in.soff = nullptr;
    in.sid = nullptr;
    in.S_owned = nullptr;
    in.Sf = nullptr;
}

// Buffers of one round.
struct RoundBufs {
    u64 tiles = 0, Pmax = 0, Tcap = 0, cap = 0, g_alloc = 0;
    u32 tp = 4096;  // positions per parse tile
    u64* string_first = nullptr;
    u64* soff_next = nullptr;
    u32* sid_next = nullptr;
    u64* R_phr = nullptr;
    u32* R_sid = nullptr;
    u32* P_slot = nullptr;
    u32* tile_cnt = nullptr;
    u64* tile_pfx = nullptr;
    u32* Tnext = nullptr;
    u32* Fnext = nullptr;
    u32* tile_str = nullptr;
    u32* brk = nullptr;
    u32* sbm = nullptr;
    u64 sbm_words = 0;
    unsigned char* tab = nullptr;  // phrase table: cap slots
    u64* rv = nullptr;             // per slot: (F^i << 32) | rank, once named
    u32* claims = nullptr;
    u32* first_bits = nullptr;
    u32* first_prefix = nullptr;
    u32* slot_r = nullptr;
    u32* len_r = nullptr;
    u64* xlen = nullptr;
    u64* mkey = nullptr;
    u64* mval = nullptr;
    u64* rkey = nullptr;
};

// The next sequence (Tnext, Fnext) gets `t_cap` entries; 0 leaves it to
// alloc_next (a round run with a host synchronisation knows its phrase count
// after the parse).
void alloc_next(lcg_ctx* ctx, RoundBufs& b, u64 t_cap) {
    b.Tcap = std::min<u64>(t_cap, b.Pmax);
    b.Tnext = dalloc<u32>(ctx, b.Tcap);
    b.Fnext = dalloc<u32>(ctx, b.Tcap);
}

// Positions per parse tile of a round of at most n symbols: the tuning's
// tile, halved (down to 1024) while the round would have fewer than
// parse_tile_min tiles per SM, so that short rounds (late rounds, small
// batches) still give every resident k_parse block several tiles.
u32 round_tile(const lcg_ctx* ctx, u64 n) {
    u32 tp = ctx->tuning.parse_tile;
    const u64 want = (u64)ctx->tuning.parse_tile_min * (u64)ctx->sms;
    while (tp > 1024 && (n + tp - 1) / tp < want) tp >>= 1;
    return tp;
}

void alloc_round(lcg_ctx* ctx, RoundBufs& b, u64 n_bound, u32 kk, u64 t_cap) {
    b.tp = round_tile(ctx, n_bound);
    b.tiles = (n_bound + b.tp - 1) / b.tp;
    // every phrase but a string's first has length >= 2
    b.Pmax = n_bound / 2 + 2ull * kk + 1;
    b.string_first = dalloc<u64>(ctx, kk);
    b.soff_next = dalloc<u64>(ctx, kk + 1);
    b.sid_next = dalloc<u32>(ctx, kk);
    b.R_phr = dalloc<u64>(ctx, kk);
    b.R_sid = dalloc<u32>(ctx, kk);
    b.P_slot = dalloc<u32>(ctx, parse_slot_entries(b.tiles, kk, b.tp));
    b.tile_cnt = dalloc<u32>(ctx, b.tiles);
    b.tile_pfx = dalloc<u64>(ctx, b.tiles);
    if (t_cap) alloc_next(ctx, b, t_cap);
    b.tile_str = dalloc<u32>(ctx, b.tiles);
    b.brk = dalloc<u32>(ctx, b.tiles * b.tp / 32);
    b.sbm_words = b.tiles * b.tp / 32 + 2;  // positions 0 .. n inclusive
    b.sbm = dalloc<u32>(ctx, b.sbm_words);
    ck(ctx, cudaMemsetAsync(b.sbm, 0, b.sbm_words * sizeof(u32), ctx->st), "memset starts");
}

void alloc_table(lcg_ctx* ctx, RoundBufs& b, u64 cap) {
    b.cap = cap;
    b.tab = dalloc<unsigned char>(ctx, cap * slot_bytes());
    b.rv = dalloc<u64>(ctx, cap);
    b.claims = dalloc<u32>(ctx, cap);
    ck(ctx, cudaMemsetAsync(b.tab, 0xFF, cap * slot_bytes(), ctx->st), "memset table");
}

void free_table(lcg_ctx* ctx, RoundBufs& b) {
    dfree(ctx, b.tab);
    dfree(ctx, b.rv);
    dfree(ctx, b.claims);
    b.tab = nullptr;
    b.rv = nullptr;
    b.claims = nullptr;
}

void alloc_naming(lcg_ctx* ctx, RoundBufs& b, u64 g_alloc) {
    b.g_alloc = g_alloc;
    const u64 nw = b.tiles * b.tp / 32;  // order keys tile * TP + q
    b.first_bits = dalloc<u32>(ctx, nw);
    b.first_prefix = dalloc<u32>(ctx, nw);
    b.slot_r = dalloc<u32>(ctx, g_alloc);
    b.len_r = dalloc<u32>(ctx, g_alloc);
    b.xlen = dalloc<u64>(ctx, g_alloc);
    b.mkey = dalloc<u64>(ctx, 2 * g_alloc);  // 16-byte keys
    b.mval = dalloc<u64>(ctx, g_alloc);
    b.rkey = dalloc<u64>(ctx, 2 * g_alloc);
    ck(ctx, cudaMemsetAsync(b.first_bits, 0, nw * sizeof(u32), ctx->st), "memset bits");
}

// Free a round's buffers except those that become the next round's input.
void free_round(lcg_ctx* ctx, RoundBufs& b) {
    for (void* p : {(void*)b.string_first, (void*)b.R_phr, (void*)b.R_sid, (void*)b.P_slot, (void*)b.tile_cnt,
                    (void*)b.tile_pfx, (void*)b.tile_str, (void*)b.brk, (void*)b.sbm, (void*)b.first_bits,
                    (void*)b.first_prefix,
                    (void*)b.slot_r, (void*)b.len_r, (void*)b.xlen, (void*)b.mkey, (void*)b.mval, (void*)b.rkey})
        dfree(ctx, p);
    free_table(ctx, b);
}

// Bits that hold every rank below `count` (at least 1).
int rank_width(u64 count) {
    int w = 1;
    while (w < 31 && (1ull << w) < count) w++;
    return w;
}

RoundArgs round_args(lcg_ctx* ctx, lcg_grammar* R, const RoundInput& in, RoundBufs& b, u32 i) {
    RoundArgs a{};
    a.sym_bytes = in.symb;
    a.sym_w = in.symb == 1 ? 8 : 31;
    a.S = in.S;
    a.Sf = in.Sf;
    a.n = in.n;
    a.d_n = in.d_n;
    a.soff = in.soff;
    a.sid = in.sid;
    a.k = in.kk;
    a.d_k = in.d_k;
    a.Fprev = fprev_of(R, i);
    a.lh = level_hash(ctx, i);
    a.level = i;
    a.parse_blocks = ctx->tuning.parse_blocks_per_sm;
    a.stripes = ctx->tuning.tile_stripes;
    a.miss_flush = ctx->tuning.miss_flush;
    a.tiles_bound = b.tiles;
    a.tp = b.tp;
    a.string_first = b.string_first;
    a.tile_str = b.tile_str;
    a.brk = b.brk;
    a.sbm = b.sbm;
    a.sbm_words = b.sbm_words;
    a.tile_cnt = b.tile_cnt;
    a.tile_pfx = b.tile_pfx;
    a.ctr = ctx->ctr;
    a.ds = ctx->ds_arr + (i - 1);
    a.rc = ctx->rc_arr + (i - 1);
    a.total = ctx->tot_arr + 3 * (i - 1);  // [0] phrases; [1], [2] scratch of the scans
    a.d_tiles = &a.rc->tiles;
    a.d_gnew = &a.ds->claims;
    a.d_Gnew = &a.ds->claim_len;
    a.soff_next = b.soff_next;
    a.sid_next = b.sid_next;
    a.R_phr = b.R_phr;
    a.R_sid = b.R_sid;
    a.P_slot = b.P_slot;
    a.T_cap = b.Tcap;
    a.Tnext = b.Tnext;
    a.Fnext = b.Fnext;
    a.c_level = R->c_level;
    a.c_rank = R->c_rank;
    return a;
}

void set_table(RoundArgs& a, RoundBufs& b) {
    a.tab = b.tab;
    a.rv = b.rv;
    a.tab_cap = b.cap;
    a.claims = b.claims;
    a.claim_limit = b.cap - b.cap / 5;
}

// Parse: tile strings, k_parse, tile scan, strings.
void enqueue_parse(lcg_ctx* ctx, RoundArgs& a, u64 n_for_bytes) {
    const Range range("parse, round", a.level);
    if (!round_is_small(a)) {
        const int ht = kt_begin(ctx, "k_tile_strings", 4.0 * (double)a.tiles_bound, a.level);
        ck(ctx, launch_tile_strings(a, ctx->st), "k_tile_strings");
        kt_end(ctx, ht);
    }
    // k_breaks' look-ahead words: a buffer of their own, so that no other
    // kernel's data can read as a head of this launch's epoch
    const u64 steps = breaks_steps(a.tiles_bound, a.tp);
    ensure_lb(ctx, &ctx->heads, &ctx->heads_steps, steps, steps * sizeof(u64));
    a.heads = reinterpret_cast<u64*>(ctx->heads);
    a.brk_epoch = ++ctx->epoch;
    if (round_is_small(a)) {
        // a short round: tile strings, breaks, parse, scan and strings in one cooperative launch
        const int hs = kt_begin(ctx, "k_parse_small", 5.0 * (double)n_for_bytes, a.level);
        const u64 bar = ctx->ctr_val;  // the grid barriers' counter values
        ctx->ctr_val += (u64)kSmallParseBarriers * small_round_grid(a);
        ck(ctx, launch_parse_small(a, bar, ctx->st), "k_parse_small");
        kt_end(ctx, hs);
        ctx->launches += 1;
        return;
    }
    int hb = kt_begin(ctx, "k_breaks", (a.sym_bytes == 1 ? 1.0 : 4.0) * n_for_bytes + (double)n_for_bytes / 8.0, a.level);
    ck(ctx, launch_breaks(a, ctx->st), "k_breaks");
    kt_end(ctx, hb);
    const double tab_bytes = a.tab_cap * (double)slot_bytes();
    const double tbytes = tab_bytes > kL2Bytes ? 32.0 * (double)n_for_bytes / 3.0 : 0.0;
    int h = kt_begin(ctx, "k_parse",
                     (a.sym_bytes == 1 ? 1.0 : 4.0) * n_for_bytes + (double)n_for_bytes / 8.0 +
                         4.0 * (double)n_for_bytes / 3.0 + tbytes, a.level);
    ck(ctx, launch_parse(a, ctx->st), "k_parse");
    kt_end(ctx, h);
    const u64 stiles = std::max<u64>(1, scan2_tiles_for(a.tiles_bound));
    ensure_lb(ctx, &ctx->lb2, &ctx->lb2_tiles, stiles, scan2_lb_bytes(stiles));
    u64 grid = 0;
    h = kt_begin(ctx, "k_scan2", 12.0 * (double)a.tiles_bound, a.level);
    ck(ctx, launch_scan2(a.tile_cnt, nullptr, a.tiles_bound, a.tile_pfx, nullptr, a.total, ctx->lb2, ++ctx->epoch,
                         ctx->ctr, ctx->ctr_val, a.ds, ctx->st, &grid, a.d_tiles),
       "scan");
    kt_end(ctx, h);
    ctx->ctr_val += grid;
    h = kt_begin(ctx, "k_strings", 40.0 * a.k, a.level);
    ck(ctx, launch_strings(a, ctx->st), "k_strings");
    kt_end(ctx, h);
    ctx->launches += 5;
}

// Naming and rewrite: mark, popcount scan, rank, length scan, rules, rewrite.
void enqueue_naming(lcg_ctx* ctx, RoundArgs& a, RoundBufs& b, double g_bytes, double G_bytes, double P_bytes) {
    const Range range("naming, round", a.level);
    a.first_bits = b.first_bits;
    a.first_prefix = b.first_prefix;
    a.slot_r = b.slot_r;
    a.len_r = b.len_r;
    a.xlen = b.xlen;
    a.mkey = b.mkey;
    a.mval = b.mval;
    a.rkey = b.rkey;
    a.g_alloc = b.g_alloc;
    const u64 g_grid = std::max<u64>(1, b.g_alloc);
    if (round_is_small(a)) {
        // a short round: marks, popcount prefix, ranks, length scan, rules and rewrite in one
        // cooperative launch
        const int hs = kt_begin(ctx, "k_naming_small", 12.0 * P_bytes, a.level);
        const u64 bar = ctx->ctr_val;
        ctx->ctr_val += (u64)kSmallNamingBarriers * small_round_grid(a);
        ck(ctx, launch_naming_small(a, b.tiles * b.tp / 32, g_grid, bar, ctx->st), "k_naming_small");
        kt_end(ctx, hs);
        ctx->launches += 1;
        return;
    }
    int h = kt_begin(ctx, "k_mark", 12.0 * g_bytes, a.level);
    ck(ctx, launch_mark(a, g_grid, ctx->st), "k_mark");
    kt_end(ctx, h);
    const u64 nw = b.tiles * b.tp / 32;
    const u64 ptiles = std::max<u64>(1, popscan_tiles_for(nw));
    ensure_lb(ctx, &ctx->lb1, &ctx->lb1_tiles, ptiles, lb1_bytes(ptiles));
    a.lb1 = ctx->lb1;
    a.epoch = ++ctx->epoch;
    a.ctr_base = ctx->ctr_val;
    ctx->ctr_val += ptiles;
    h = kt_begin(ctx, "k_popscan", 8.0 * (double)nw, a.level);
    ck(ctx, launch_popscan(a, nw, ctx->st), "k_popscan");
    kt_end(ctx, h);
    h = kt_begin(ctx, "k_rank", 24.0 * g_bytes, a.level);
    ck(ctx, launch_rank(a, g_grid, ctx->st), "k_rank");
    kt_end(ctx, h);
    const u64 stiles = std::max<u64>(1, scan2_tiles_for(g_grid));
    ensure_lb(ctx, &ctx->lb2, &ctx->lb2_tiles, stiles, scan2_lb_bytes(stiles));
    u64 grid = 0;
    h = kt_begin(ctx, "k_scan2", 12.0 * g_bytes, a.level);
    ck(ctx, launch_scan2(b.len_r, nullptr, g_grid, b.xlen, nullptr, a.total + 1, ctx->lb2, ++ctx->epoch, ctx->ctr,
                         ctx->ctr_val, a.ds, ctx->st, &grid, a.d_gnew),
       "scan");
    kt_end(ctx, h);
    ctx->ctr_val += grid;
    h = kt_begin(ctx, "k_rules", 4.0 * G_bytes + 12.0 * g_bytes, a.level);
    ck(ctx, launch_rules(a, g_grid, ctx->st), "k_rules");
    kt_end(ctx, h);
    h = kt_begin(ctx, "k_rewrite", 12.0 * P_bytes, a.level);
    ck(ctx, launch_rewrite(a, ctx->st), "k_rewrite");
    kt_end(ctx, h);
    ctx->launches += 6;
}

void next_input(lcg_ctx* ctx, RoundInput& in, RoundBufs& b) {
    if (in.own_offsets) {
        dfree(ctx, in.soff);
        dfree(ctx, in.sid);
    }
    in.own_offsets = true;
    if (in.S_owned) dfree(ctx, in.S_owned);
    if (in.Sf) dfree(ctx, (void*)in.Sf);
    in.S = b.Tnext;
    in.S_owned = b.Tnext;
    in.Sf = b.Fnext;
    in.symb = 4;
    in.soff = b.soff_next;
    in.sid = b.sid_next;
}

// One round with a host synchronisation after the parse: the table is
// regrown and the parse rerun until it fits, and all later sizes are exact.
void round_sync(lcg_ctx* ctx, lcg_grammar* R, RoundInput& in, u32 i, bool against_resident, double& prev_ratio,
                double& p_ratio) {
    fail_if(ctx, i >= ctx->levels || i > kMaxRounds,
            LCG_ELEVELS, "hash family too short: needs more than " + std::to_string(ctx->levels) + " functions");
    if (R->lv.size() < i) R->lv.emplace_back();
    lcg_round_stats& rs = ctx->stats.round[std::min<u32>(i - 1, 63)];
    const u64 n = in.n;
    rs.n = n;
    rs.strings = in.kk;
    RoundBufs b;
    alloc_round(ctx, b, n, in.kk, 0);
    const u64 tiles = b.tiles;
    ensure_lb(ctx, &ctx->lb1, &ctx->lb1_tiles, tiles, lb1_bytes(tiles));
    Level& L = R->lv[i - 1];
    RoundArgs a = round_args(ctx, R, in, b, i);
    a.d_n = nullptr;
    a.d_k = nullptr;
    // inline keys as narrow as the level below allows; tables of resident
    // grammars keep the full width
    if (i > 1 && !against_resident) a.sym_w = rank_width(R->lv[i - 2].g);
    if (against_resident && L.g > 0) {
        ensure_resident(ctx, R, i, L.g);
        a.rtab = L.rtab;
        a.rtab_cap = L.rcap;
        a.rrhs = L.rhs;
        a.rrhs_off = L.rhs_off;
    }
    // Phrase table: sized from the distinct/phrase ratio of this level in the
    // context's previous build when there is one (at the tuning's load, 0.5 by
    // default: short probe sequences), else from a generous guess; an
    // overflowing table is regrown and the parse rerun.
    const double hint = ctx->ratio_hint[std::min<u32>(i, 63)];
    u64 cap;
    if (hint > 0) {
        const u64 P_est = std::min<u64>(b.Pmax, (u64)(ctx->p_hint[std::min<u32>(i, 63)] * (double)n) + 64);
        cap = std::max<u64>(8192, (u64)(hint * (double)P_est / ctx->tuning.table_load) + 1024);
    } else {
        const u64 P_est = std::min<u64>(b.Pmax, (u64)(p_ratio * 1.2 * (double)n) + 64);
        const double ratio = (i == 1) ? 0.02 : std::min(1.0, std::max(prev_ratio * 2.0, 0.05));
        cap = 2 * std::max<u64>(4096, std::min<u64>(P_est, (u64)(ratio * 1.3 * (double)P_est) + 1));
    }
    if (ctx->tuning.table_slots_max) cap = std::min<u64>(cap, ctx->tuning.table_slots_max);
    u32 retries = 0;
    DevStatus st;
    RoundCounts rc;
    while (true) {
        fail_if(ctx, cap > (kMaxRank + 1), LCG_ETABLE, "phrase table would exceed 2^31 slots");
        alloc_table(ctx, b, cap);
        ck(ctx, cudaMemsetAsync(a.ds, 0, sizeof(DevStatus), ctx->st), "reset counters");
        set_table(a, b);
        enqueue_parse(ctx, a, n);
        ck(ctx, cudaMemcpyAsync(&rc, a.rc, sizeof(rc), cudaMemcpyDeviceToHost, ctx->st), "read counts");
        ck(ctx, cudaMemcpyAsync(&st, a.ds, sizeof(st), cudaMemcpyDeviceToHost, ctx->st), "read status");
        sync(ctx);
        check_device_status(ctx, st);
        if (!st.overflow) break;
        free_table(ctx, b);
        cap *= 4;
        retries++;
    }
    const u64 P = rc.phrases;
    rs.phrases = P;
    fail_if(ctx, P > b.Pmax, LCG_EDEVICE, "round produced more phrases than its bound");
    p_ratio = n ? (double)P / (double)n : 0.35;
    rs.table_cap = cap;
    rs.retries = retries;
    const u64 g_new = st.claims, G_new = st.claim_len;
    fail_if(ctx, L.g + g_new > kMaxRank, LCG_EOVERFLOW, "level with 2^31 rules or more");
    rs.g = g_new;
    rs.G = G_new;
    prev_ratio = P ? (double)g_new / (double)P : 0.0;
    record_hints(ctx, i, n, P, g_new, G_new);
    grow_level(ctx, L, L.g + g_new, L.G + G_new);
    if (against_resident) {
        ensure_resident(ctx, R, i, L.g + g_new);
        a.rtab_w = L.rtab;
        a.rtab_w_cap = L.rcap;
    } else {
        L.rvalid = false;
    }
    alloc_naming(ctx, b, g_new);
    alloc_next(ctx, b, P + 1);  // the next sequence: exactly the round's phrases
    a.Tnext = b.Tnext;
    a.Fnext = b.Fnext;
    a.T_cap = b.Tcap;
    a.g_base = L.g;
    a.G_base = L.G;
    a.cap_g = L.cap_g;
    a.cap_G = L.cap_G;
    a.rhs = L.rhs;
    a.rhs_off = L.rhs_off;
    a.F = L.F;
    enqueue_naming(ctx, a, b, (double)g_new, (double)G_new, (double)P);
    L.g += g_new;
    L.G += G_new;
    free_round(ctx, b);
    next_input(ctx, in, b);
    in.n = rc.n_next;
    in.kk = (u32)rc.k_next;
    ctx->stats.rounds = i;
}

// Sizes of the rounds of a build enqueued without host synchronisation,
// planned from the context's hints (new rules per phrase, phrases per symbol,
// symbols per rule of each level) and its plan slack.
struct RoundPlan {
    u64 n_bound = 0, n_est = 0, n_alloc = 0, cap = 0, g_alloc = 0, G_alloc = 0, t_cap = 0;
    double P_est = 0, g_est = 0, G_est = 0;
};

// x rounded up to a step of 2^(1/4) (about 19 %): plans from slightly
// different hints get the same buffers, so a captured graph can be reused.
u64 bucket(u64 x) {
    if (x <= 16) return x;
    const int e = 63 - __builtin_clzll(x);
    const u64 b = 1ull << e;
    for (const double f : {1.0, 1.189207115, 1.414213562, 1.681792831, 2.0}) {
        const u64 v = (u64)std::ceil((double)b * f);
        if (v >= x) return v;
    }
    return 2 * b;
}

std::vector<RoundPlan> plan_rounds(lcg_ctx* ctx, u64 n1, u32 kk, u32 planned) {
    std::vector<RoundPlan> v(planned + 1);
    u64 n_bound = n1, n_est = n1;
    for (u32 r = 1; r <= planned; r++) {
        RoundPlan& p = v[r];
        p.n_bound = n_bound;
        p.n_est = n_est;
        // the round's sequence is at most the planned next sequence of the
        // round before (which flags a capacity error past it)
        p.n_alloc = (r == 1) ? n_bound : std::min<u64>(n_bound, v[r - 1].t_cap);
        p.P_est = ctx->p_hint[r] * (double)n_est;
        p.g_est = ctx->ratio_hint[r] * p.P_est;
        p.G_est = ctx->glen_hint[r] * p.g_est;
        // slack over the estimates: 10-25 % times the context's plan slack,
        // which grows after a plan that did not fit and shrinks while plans fit
        const double sl = ctx->plan_slack;
        p.cap = std::min<u64>(bucket(std::max<u64>(8192, (u64)(p.g_est * 1.1 * sl / ctx->tuning.table_load) + 1024)),
                              kMaxRank + 1);
        if (ctx->tuning.table_slots_max) p.cap = std::min<u64>(p.cap, ctx->tuning.table_slots_max);
        p.g_alloc = bucket((u64)(p.g_est * 1.25 * sl) + 1024);
        p.G_alloc = bucket((u64)(p.G_est * 1.25 * sl) + 4096);
        // the next sequence: the estimated phrases with the same slack (a
        // round past it flags a capacity error and the build is redone)
        p.t_cap = std::min<u64>(bucket((u64)(p.P_est * 1.1 * sl) + 4096), n_bound / 2 + 2ull * kk + 1);
        n_bound = n_bound / 2 + 2ull * kk + 1;  // every phrase but a string's first has length >= 2
        n_est = (u64)p.P_est + 64;
    }
    return v;
}

// Rounds enqueued without host synchronisation, between their enqueueing and
// the reading of their statuses.
struct AsyncRounds {
    u32 planned = 0, kk = 0;
    std::vector<RoundPlan> plan;
    std::vector<u64> g_base, G_base;
};

// Enqueue the planned rounds of a fresh build: every size comes from the plan;
// kernels read the actual sizes from the device and flag a round that
// outgrows its buffers.
void rounds_async_enqueue(lcg_ctx* ctx, lcg_grammar* R, RoundInput& in, AsyncRounds& ar) {
    const u32 planned = ar.planned;
    const u32 kk = ar.kk;
    ar.g_base.assign(planned + 1, 0);
    ar.G_base.assign(planned + 1, 0);
    for (u32 r = 1; r <= planned; r++) {
        const RoundPlan& p = ar.plan[r];
        if (R->lv.size() < r) R->lv.emplace_back();
        Level& L = R->lv[r - 1];
        RoundBufs b;
        alloc_round(ctx, b, p.n_alloc, kk, p.t_cap);
        ensure_lb(ctx, &ctx->lb1, &ctx->lb1_tiles, b.tiles, lb1_bytes(b.tiles));
        RoundArgs a = round_args(ctx, R, in, b, r);
        // a round stops early when the one before it failed
        if (r > 1) a.ds_prev = ctx->ds_arr + (r - 2);
        // every rank of the level below is under its capacity
        if (r > 1) a.sym_w = rank_width(R->lv[r - 2].cap_g);
        alloc_table(ctx, b, p.cap);
        set_table(a, b);
        enqueue_parse(ctx, a, p.n_est);
        grow_level(ctx, L, L.g + p.g_alloc, L.G + p.G_alloc);
        L.rvalid = false;
        alloc_naming(ctx, b, p.g_alloc);
        ar.g_base[r] = L.g;
        ar.G_base[r] = L.G;
        a.g_base = L.g;
        a.G_base = L.G;
        a.cap_g = L.cap_g;
        a.cap_G = L.cap_G;
        a.rhs = L.rhs;
        a.rhs_off = L.rhs_off;
        a.F = L.F;
        enqueue_naming(ctx, a, b, p.g_est, p.G_est, p.P_est);
        free_round(ctx, b);
        next_input(ctx, in, b);
        in.d_n = &a.rc->n_next;
        in.d_k = &a.rc->k_next;
    }
}

// After the enqueued rounds: read their statuses and counts (one host
// synchronisation), set the levels' sizes and the build statistics.  Returns
// 0, or -1 when a round did not fit (the build must then be redone round by
// round); `i` becomes the first round not yet run, and `in` its input.
int rounds_async_finish(lcg_ctx* ctx, lcg_grammar* R, RoundInput& in, const AsyncRounds& ar, u32& i) {
    const u32 planned = ar.planned;
    const u32 kk = ar.kk;
    std::vector<DevStatus> st(planned);
    std::vector<RoundCounts> rc(planned);
    ck(ctx, cudaMemcpyAsync(st.data(), ctx->ds_arr, planned * sizeof(DevStatus), cudaMemcpyDeviceToHost, ctx->st),
       "read status");
    ck(ctx, cudaMemcpyAsync(rc.data(), ctx->rc_arr, planned * sizeof(RoundCounts), cudaMemcpyDeviceToHost, ctx->st),
       "read counts");
    sync(ctx);
    for (u32 r = 0; r < planned; r++) {
        if (st[r].overflow || st[r].error == kErrCapacity || st[r].error == kErrHalted) return -1;
        check_device_status(ctx, st[r]);
    }
    // rounds past the last active string (the data needed fewer rounds than
    // the previous build) leave empty levels: drop them
    u32 used = planned;
    for (u32 r = 1; r <= planned; r++) {
        const u64 k_in = (r == 1) ? kk : rc[r - 2].k_next;
        if (k_in == 0) { used = r - 1; break; }
    }
    while (R->lv.size() > used && R->lv.back().g == 0 && ar.g_base.size() > R->lv.size()) {
        Level& L = R->lv.back();
        if (st[R->lv.size() - 1].claims != 0) break;
        dfree(ctx, L.rhs_off);
        dfree(ctx, L.rhs);
        dfree(ctx, L.F);
        dfree(ctx, L.rtab);
        R->lv.pop_back();
    }
    u64 n = in.n;
    for (u32 r = 1; r <= used; r++) {
        Level& L = R->lv[r - 1];
        const DevStatus& s = st[r - 1];
        const RoundCounts& c = rc[r - 1];
        fail_if(ctx, L.g + s.claims > kMaxRank, LCG_EOVERFLOW, "level with 2^31 rules or more");
        L.g = ar.g_base[r] + s.claims;
        L.G = ar.G_base[r] + s.claim_len;
        lcg_round_stats& rs = ctx->stats.round[r - 1];
        rs.n = n;
        rs.strings = (r == 1) ? kk : rc[r - 2].k_next;
        rs.phrases = c.phrases;
        rs.table_cap = ar.plan[r].cap;
        rs.g = s.claims;
        rs.G = s.claim_len;
        record_hints(ctx, r, n, c.phrases, s.claims, s.claim_len);
        n = c.n_next;
        ctx->stats.rounds = r;
    }
    ctx->stats.async_rounds = used;
    in.n = rc[planned - 1].n_next;
    in.kk = (u32)rc[planned - 1].k_next;
    in.d_n = nullptr;
    in.d_k = nullptr;
    i = planned + 1;
    return 0;
}

u32 planned_rounds(const lcg_ctx* ctx) {
    return std::min<u32>(ctx->hint_rounds, std::min<u32>(ctx->levels - 1, kMaxRounds));
}

// The rounds of a fresh build, enqueued without host synchronisation and
// planned from the context's previous builds.
int rounds_async(lcg_ctx* ctx, lcg_grammar* R, RoundInput& in, u32& i) {
    AsyncRounds ar;
    ar.planned = planned_rounds(ctx);
    ar.kk = in.kk;
    ar.plan = plan_rounds(ctx, in.n, in.kk, ar.planned);
    rounds_async_enqueue(ctx, R, in, ar);
    return rounds_async_finish(ctx, R, in, ar, i);
}

// ---- the rounds of a build as one CUDA graph ------------------------------
//
// A context's builds of one shape (the same device input buffer, string
// lengths and plan) can run as one captured graph: the first such build
// captures every round's allocations, memsets and launches (the planned
// rounds, as enqueued without host synchronisation), later builds launch it.
// The graph writes the grammar into its own allocations, which keep their
// addresses at every launch: a launch therefore waits until the grammar of
// the previous launch has been freed (a serving loop's build -> use -> free),
// and otherwise the build runs as launches.  The graph resets the single-pass
// tile counter and the look-back flags it uses; the string offsets of round 1
// are uploaded to buffers outside the graph before each launch.

struct GraphBuild {
    // what the launches depend on
    const unsigned char* d_in = nullptr;
    u64 n1 = 0;
    u32 k = 0;
    std::vector<u64> lens;
    std::vector<double> params;  // planned rounds and launch parameters (graph_params)
    // round-1 offsets and ids, outside the graph
    u64* soff = nullptr;
    u32* sid = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    lcg_grammar shape;  // host description of the grammar a launch writes
    AsyncRounds ar;
    u64 ctr_end = 0;    // tile counter after a launch
    u64 launches = 0;   // kernels per launch
    std::vector<lcg_ctx::KRec> krecs;  // timing events recorded by the graph
    lcg_grammar* live = nullptr;       // grammar of the last launch, until freed
};

// What a graph's launches depend on besides the input and the planned buffer
// sizes: the number of planned rounds and the launch parameters.
std::vector<double> graph_params(lcg_ctx* ctx, u32 planned) {
    return {(double)planned,    (double)ctx->tuning.parse_blocks_per_sm, (double)ctx->tuning.miss_flush,
            (double)ctx->ktime, (double)ctx->tuning.tile_stripes,        (double)ctx->tuning.parse_tile,
            (double)ctx->tuning.parse_tile_min};
}

// A captured graph serves a new plan when each of its rounds' buffers holds
// the new plan's (the kernels read the actual sizes from the device, so a
// larger buffer changes nothing but memory), and its phrase tables are not
// more than 4x the new plan's (a table far larger than needed costs its
// clearing and L2 room).  Hints that decay and a plan slack that shrinks
// after every build that fits therefore keep the graph; a plan that grows
// past it, or shrinks far below it, captures a new one.
bool plan_covers(const std::vector<RoundPlan>& have, const std::vector<RoundPlan>& need) {
    if (have.size() != need.size()) return false;
    for (size_t r = 1; r < have.size(); r++) {
        const RoundPlan& h = have[r];
        const RoundPlan& n = need[r];
        if (h.n_bound != n.n_bound || h.n_alloc < n.n_alloc || h.cap < n.cap || h.cap > 4 * n.cap ||
            h.g_alloc < n.g_alloc || h.G_alloc < n.G_alloc || h.t_cap < n.t_cap)
            return false;
    }
    return true;
}

void destroy_graph(lcg_ctx* ctx) {
    GraphBuild* gb = ctx->graph;
    if (!gb) return;
    cudaStreamSynchronize(ctx->st);
    if (gb->exec) cudaGraphExecDestroy(gb->exec);
    if (gb->graph) cudaGraphDestroy(gb->graph);
    // the records of the last launch name the graph's events: they go with them
    ctx->krecs.erase(std::remove_if(ctx->krecs.begin(), ctx->krecs.end(),
                                    [](const lcg_ctx::KRec& r) { return r.graph; }),
                     ctx->krecs.end());
    for (auto& r : gb->krecs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    if (gb->soff) cudaFreeAsync(gb->soff, ctx->st);
    if (gb->sid) cudaFreeAsync(gb->sid, ctx->st);
    // a live grammar of the graph keeps its memory (freed with the grammar);
    // the rest of the graph's memory goes back to the device now, not when
    // another graph would reuse it
    delete gb;
    ctx->graph = nullptr;
    cudaStreamSynchronize(ctx->st);
    cudaDeviceGraphMemTrim(ctx->device);
}

void graph_grammar_freed(lcg_ctx* ctx, const lcg_grammar* G) {
    if (ctx->graph && ctx->graph->live == G) ctx->graph->live = nullptr;
}

// Capture the planned rounds of a build of this shape (nothing runs yet).
void capture_graph(lcg_ctx* ctx, const unsigned char* d_in, const std::vector<u64>& lens, u32 planned,
                   std::vector<double> params) {
    destroy_graph(ctx);
    const u32 k = (u32)lens.size();
    u64 n1 = 0;
    for (u64 x : lens) n1 += x;
    std::vector<RoundPlan> plan = plan_rounds(ctx, n1, k, planned);
    // look-back buffers and timing events for every launch, made before the
    // capture (the graph must not reallocate them)
    u64 t1 = 1, t2 = 1, hs = 1;
    for (u32 r = 1; r <= planned; r++) {
        const RoundPlan& p = plan[r];
        const u32 tp = round_tile(ctx, p.n_alloc);
        const u64 tiles = (p.n_alloc + tp - 1) / tp;
        t1 = std::max({t1, tiles, popscan_tiles_for(tiles * tp / 32)});
        t2 = std::max({t2, scan2_tiles_for(tiles), scan2_tiles_for(std::max<u64>(1, p.g_alloc))});
        hs = std::max(hs, breaks_steps(tiles, tp));
    }
    ensure_lb(ctx, &ctx->lb1, &ctx->lb1_tiles, t1, lb1_bytes(t1));
    ensure_lb(ctx, &ctx->lb2, &ctx->lb2_tiles, t2, scan2_lb_bytes(t2));
    ensure_lb(ctx, &ctx->heads, &ctx->heads_steps, hs, hs * sizeof(u64));
    auto* gb = new GraphBuild;
    ctx->graph = gb;
    gb->d_in = d_in;
    gb->k = k;
    gb->lens = lens;
    gb->params = std::move(params);
    gb->n1 = n1;
    gb->soff = dalloc<u64>(ctx, k + 1);
    gb->sid = dalloc<u32>(ctx, k);
    gb->ar.planned = planned;
    gb->ar.kk = k;
    gb->ar.plan = std::move(plan);
    if (ctx->ktime)
        while (ctx->evpool.size() < 24ull * planned + 8) {
            cudaEvent_t e;
            ck(ctx, cudaEventCreate(&e), "cudaEventCreate");
            ctx->evpool.push_back(e);
        }
    sync(ctx);
    const size_t krec0 = ctx->krecs.size();
    const u64 launches0 = ctx->launches;
    const u64 ctr_before = ctx->ctr_val;  // the device counter until the graph runs
    ck(ctx, cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal), "begin capture");
    ctx->capturing = true;
    lcg_grammar* T = nullptr;
    try {
        ck(ctx, cudaMemsetAsync(ctx->ctr, 0, sizeof(u64), ctx->st), "reset tile counter");
        ctx->ctr_val = 0;
        ck(ctx, cudaMemsetAsync(ctx->lb1, 0, lb1_bytes(ctx->lb1_tiles), ctx->st), "reset look-back");
        // the graph's launches reuse its epochs: heads of the last launch must not read as published
        ck(ctx, cudaMemsetAsync(ctx->heads, 0, ctx->heads_steps * sizeof(u64), ctx->st), "reset heads");
        ck(ctx, cudaMemsetAsync(ctx->lb2, 0, scan2_lb_bytes(ctx->lb2_tiles), ctx->st), "reset look-back");
        T = new_grammar(ctx, false);
        grow_c(ctx, T, k);
        T->k = k;
        ck(ctx, cudaMemsetAsync(ctx->ds_arr, 0, kMaxRounds * sizeof(DevStatus), ctx->st), "reset status");
        ck(ctx, cudaMemsetAsync(ctx->rc_arr, 0, kMaxRounds * sizeof(RoundCounts), ctx->st), "reset counts");
        RoundInput in{};
        in.S = d_in;
        in.symb = 1;
        in.n = gb->n1;
        in.kk = k;
        in.soff = gb->soff;
        in.sid = gb->sid;
        in.own_offsets = false;
        rounds_async_enqueue(ctx, T, in, gb->ar);
        free_round_input(ctx, in);  // the last round's outputs: the graph's own allocations
    } catch (...) {
        ctx->capturing = false;
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(ctx->st, &g);
        if (g) cudaGraphDestroy(g);
        delete T;
        ctx->ctr_val = ctr_before;
        destroy_graph(ctx);
        throw;
    }
    ctx->capturing = false;
    const cudaError_t e = cudaStreamEndCapture(ctx->st, &gb->graph);
    gb->ctr_end = ctx->ctr_val;
    ctx->ctr_val = ctr_before;
    if (e != cudaSuccess) {
        delete T;
        destroy_graph(ctx);
        ck(ctx, e, "end capture");
    }
    gb->shape = *T;
    delete T;  // host object only: its device arrays are the graph's allocations
    gb->launches = ctx->launches - launches0;
    for (size_t x = krec0; x < ctx->krecs.size(); x++) {
        gb->krecs.push_back(ctx->krecs[x]);
        gb->krecs.back().graph = true;
    }
    ctx->krecs.resize(krec0);
    const cudaError_t ei = cudaGraphInstantiate(&gb->exec, gb->graph, 0);
    if (ei != cudaSuccess) {
        destroy_graph(ctx);
        ck(ctx, ei, "instantiate graph");
    }
}

// A build as a launch of the context's graph (captured first when the shape
// is new).  Returns the grammar, or nullptr when the build must run as
// launches (the graph's last grammar is still in use); throws Retry when the
// planned rounds did not fit.
lcg_grammar* build_with_graph(lcg_ctx* ctx, const unsigned char* d_in, const std::vector<u64>& lens) {
    const u32 k = (u32)lens.size();
    const u32 planned = planned_rounds(ctx);
    u64 n1 = 0;
    for (u64 x : lens) n1 += x;
    std::vector<double> params = graph_params(ctx, planned);
    GraphBuild* gb = ctx->graph;
    const bool same = gb && gb->d_in == d_in && gb->lens == lens && gb->params == params &&
                      plan_covers(gb->ar.plan, plan_rounds(ctx, n1, k, planned));
    if (same && gb->live) return nullptr;
    const u32 mode = same ? 2 : 1;
    if (!same) {
        capture_graph(ctx, d_in, lens, planned, std::move(params));
        gb = ctx->graph;
    }
    std::vector<u64> soff_h(k + 1, 0);
    std::vector<u32> sid_h(k);
    for (u32 j = 0; j < k; j++) {
        soff_h[j + 1] = soff_h[j] + lens[j];
        sid_h[j] = j;
    }
    ctx->stats = lcg_build_stats{};
    ctx->stats.input_bytes = gb->n1;
    ck(ctx, cudaMemcpyAsync(gb->soff, soff_h.data(), (k + 1) * sizeof(u64), cudaMemcpyHostToDevice, ctx->st),
       "upload offsets");
    ck(ctx, cudaMemcpyAsync(gb->sid, sid_h.data(), k * sizeof(u32), cudaMemcpyHostToDevice, ctx->st), "upload ids");
    ck(ctx, cudaGraphLaunch(gb->exec, ctx->st), "graph launch");
    ctx->ctr_val = gb->ctr_end;
    ctx->launches += gb->launches;
    for (const auto& r : gb->krecs) ctx->krecs.push_back(r);
    lcg_grammar* G = new lcg_grammar(gb->shape);
    G->owner = ctx;
    ctx->live.push_back(G);
    gb->live = G;
    RoundInput in{};
    in.n = gb->n1;
    in.kk = k;
    u32 i = 0;
    int r;
    try {
        r = rounds_async_finish(ctx, G, in, gb->ar, i);
    } catch (...) {
        free_grammar_now(G);
        throw;
    }
    if (r < 0 || in.kk > 0) {  // did not fit, or more rounds are needed: run as launches
        free_grammar_now(G);
        throw Retry{};
    }
    ctx->hint_rounds = ctx->stats.rounds;
    ctx->stats.kernel_launches = gb->launches;
    ctx->stats.graph = mode;
    return G;
}

void build_into(lcg_ctx* ctx, lcg_grammar* R, const uint8_t* data, const uint64_t* off, uint32_t k, int on_dev,
                bool against_resident, bool allow_async) {
    fail_if(ctx, k == 0 || off == nullptr || data == nullptr, LCG_EINVAL, "empty collection");
    fail_if(ctx, (u64)R->k + k > 0xffffffffull, LCG_EOVERFLOW, "too many strings");
    std::vector<u64> act_src, act_len, lvl0_pos;
    std::vector<u32> act_id, lvl0_id;
    for (u32 j = 0; j < k; j++) {
        fail_if(ctx, off[j + 1] <= off[j], LCG_EINVAL, "string " + std::to_string(j) + " is empty");
        const u64 len = off[j + 1] - off[j];
        if (len == 1) {
            lvl0_pos.push_back(off[j] - off[0]);
            lvl0_id.push_back(R->k + j);
        } else {
            act_src.push_back(off[j] - off[0]);
            act_len.push_back(len);
            act_id.push_back(R->k + j);
        }
    }
    ctx->stats = lcg_build_stats{};
    ctx->stats.input_bytes = off[k] - off[0];
    const u64 launches0 = ctx->launches;
    std::vector<void*> owned;  // freed at the end
    auto own = [&](void* p) { owned.push_back(p); return p; };

    const u64 nbytes = off[k] - off[0];
    const unsigned char* d_in;
    if (on_dev) {
        d_in = data + off[0];
    } else {
        unsigned char* p = dalloc<unsigned char>(ctx, nbytes);
        own(p);
        ck(ctx, cudaMemcpyAsync(p, data + off[0], nbytes, cudaMemcpyHostToDevice, ctx->st), "copy input");
        d_in = p;
    }
    const u32 kbase = R->k;
    grow_c(ctx, R, R->k + k);
    R->k += k;

    if (!lvl0_id.empty()) {
        u64* dpos = (u64*)own(dalloc<u64>(ctx, lvl0_pos.size()));
        u32* dids = (u32*)own(dalloc<u32>(ctx, lvl0_id.size()));
        ck(ctx, cudaMemcpyAsync(dpos, lvl0_pos.data(), lvl0_pos.size() * 8, cudaMemcpyHostToDevice, ctx->st), "copy");
        ck(ctx, cudaMemcpyAsync(dids, lvl0_id.data(), lvl0_id.size() * 4, cudaMemcpyHostToDevice, ctx->st), "copy");
        ck(ctx, launch_level0(d_in, dpos, dids, (u32)lvl0_id.size(), R->c_level, R->c_rank, ctx->st), "level0");
        ctx->launches++;
    }
    (void)kbase;
    u32 kk = (u32)act_id.size();
    if (kk == 0) {
        sync(ctx);
        for (void* p : owned) dfree(ctx, p);
        ctx->stats.kernel_launches = ctx->launches - launches0;
        return;
    }
    // round-1 sequence: the active strings back to back
    std::vector<u64> soff_h(kk + 1, 0);
    for (u32 x = 0; x < kk; x++) soff_h[x + 1] = soff_h[x] + act_len[x];
    const u64 n1 = soff_h[kk];
    u64* d_soff = dalloc<u64>(ctx, kk + 1);
    u32* d_sid = dalloc<u32>(ctx, kk);
    ck(ctx, cudaMemcpyAsync(d_soff, soff_h.data(), (kk + 1) * 8, cudaMemcpyHostToDevice, ctx->st), "copy soff");
    ck(ctx, cudaMemcpyAsync(d_sid, act_id.data(), kk * 4, cudaMemcpyHostToDevice, ctx->st), "copy sid");
    const void* S = d_in;
    void* S_owned = nullptr;
    if (!lvl0_id.empty()) {
        unsigned char* g = dalloc<unsigned char>(ctx, n1);
        u64* dsrc = (u64*)own(dalloc<u64>(ctx, kk));
        ck(ctx, cudaMemcpyAsync(dsrc, act_src.data(), kk * 8, cudaMemcpyHostToDevice, ctx->st), "copy");
        ck(ctx, launch_gather_strings(d_in, dsrc, d_soff, kk, g, ctx->st), "gather");
        ctx->launches++;
        S = g;
        S_owned = g;
    }
    RoundInput in{};
    in.S = S;
    in.S_owned = S_owned;
    in.Sf = nullptr;
    in.symb = 1;
    in.n = n1;
    in.kk = kk;
    in.soff = d_soff;
    in.sid = d_sid;
    ck(ctx, cudaMemsetAsync(ctx->ds_arr, 0, kMaxRounds * sizeof(DevStatus), ctx->st), "reset status");
    ck(ctx, cudaMemsetAsync(ctx->rc_arr, 0, kMaxRounds * sizeof(RoundCounts), ctx->st), "reset counts");
    u32 i = 1;
    if (allow_async && !against_resident && ctx->hint_rounds > 0) {
        const int r = rounds_async(ctx, R, in, i);
        if (r < 0) {
            // a round outgrew its estimate: the caller starts again with synchronised rounds
            free_round_input(ctx, in);
            for (void* p : owned) dfree(ctx, p);
            throw Retry{};
        }
    }
    double prev_ratio = 0.0, p_ratio = 0.35;
    for (; in.kk > 0; i++) round_sync(ctx, R, in, i, against_resident, prev_ratio, p_ratio);
    check_device_status(ctx, read_status(ctx));
    ctx->hint_rounds = ctx->stats.rounds;
    free_round_input(ctx, in);
    for (void* p : owned) dfree(ctx, p);
    ctx->stats.kernel_launches = ctx->launches - launches0;
}

// --------------------------------------------------------------------------
// MergeGrams
// --------------------------------------------------------------------------

void merge(lcg_ctx* ctx, lcg_grammar* A, const lcg_grammar* B) {
    fail_if(ctx, A == B, LCG_EINVAL, "cannot merge a grammar into itself");
    fail_if(ctx, A->tag != B->tag || A->tag != ctx->tag, LCG_EMISMATCH, "grammars of different hash families");
    fail_if(ctx, (u64)A->k + B->k > 0xffffffffull, LCG_EOVERFLOW, "too many strings");
    const u32 kb = B->k;
    u32* cb_rank = dalloc<u32>(ctx, kb);
    if (kb)
        ck(ctx, cudaMemcpyAsync(cb_rank, B->c_rank, kb * 4, cudaMemcpyDeviceToDevice, ctx->st), "copy");
    u32* Mprev = nullptr;
    for (u32 i = 1; i <= B->lv.size(); i++) {
        if (A->lv.size() < i) A->lv.emplace_back();
        Level& LA = A->lv[i - 1];
        const Level& LB = B->lv[i - 1];
        const u64 gb = LB.g;
        const u32* brhs = LB.rhs;
        u32* brhs_tmp = nullptr;
        if (i > 1 && LB.G > 0) {
            brhs_tmp = dalloc<u32>(ctx, LB.G);
            ck(ctx, launch_remap(LB.rhs, LB.G, Mprev, brhs_tmp, ctx->st), "remap");
            ctx->launches++;
            brhs = brhs_tmp;
        }
        if (LA.rhs_off == nullptr) grow_level(ctx, LA, 0, 0);
        ensure_resident(ctx, A, i, LA.g + gb);
        u32* M = dalloc<u32>(ctx, gb);
        u32* miss = dalloc<u32>(ctx, gb);
        u32* mlen = dalloc<u32>(ctx, gb);
        u64* xrank = dalloc<u64>(ctx, gb);
        u64* xlen = dalloc<u64>(ctx, gb);
        ck(ctx, launch_merge_lookup(brhs, LB.rhs_off, LB.F, gb, i == 1, fprev_of(A, i), level_hash(ctx, i), LA.rtab,
                                    LA.rcap, LA.rhs, LA.rhs_off, LA.F, M, miss, mlen, ctx->ds, ctx->st),
           "merge lookup");
        u64 grid = 0;
        const u64 stiles = std::max<u64>(1, scan2_tiles_for(gb));
        ensure_lb(ctx, &ctx->lb2, &ctx->lb2_tiles, stiles, scan2_lb_bytes(stiles));
        ck(ctx, launch_scan2(miss, mlen, gb, xrank, xlen, ctx->scratch + 1, ctx->lb2, ++ctx->epoch, ctx->ctr,
                             ctx->ctr_val, ctx->ds, ctx->st, &grid),
           "scan");
        ctx->ctr_val += grid;
        ctx->launches += 2;
        u64 tot[2] = {0, 0};
        if (gb) ck(ctx, cudaMemcpyAsync(tot, ctx->scratch + 1, 16, cudaMemcpyDeviceToHost, ctx->st), "read totals");
        check_device_status(ctx, read_status(ctx));
        const u64 ga = LA.g, Ga = LA.G;
        fail_if(ctx, ga + tot[0] > kMaxRank, LCG_EOVERFLOW, "level with 2^31 rules or more");
        grow_level(ctx, LA, ga + tot[0], Ga + tot[1]);
        ck(ctx, launch_merge_append(brhs, LB.rhs_off, LB.F, gb, miss, xrank, xlen, ga, Ga, LA.rhs, LA.rhs_off, LA.F,
                                    M, ga + tot[0], Ga + tot[1], ctx->st),
           "merge append");
        ctx->launches += 2;
        LA.g = ga + tot[0];
        LA.G = Ga + tot[1];
        // the appended rules join the table of the level
        ck(ctx, launch_resident_build(LA.rhs, LA.rhs_off, ga, tot[0], i == 1, fprev_of(A, i), level_hash(ctx, i),
                                      LA.rtab, LA.rcap, ctx->ds, ctx->st),
           "table insert");
        ck(ctx, launch_remap_c(B->c_level, cb_rank, kb, i, M, ctx->st), "remap C");
        ctx->launches += 2;
        dfree(ctx, brhs_tmp);
        dfree(ctx, miss);
        dfree(ctx, mlen);
        dfree(ctx, xrank);
        dfree(ctx, xlen);
        dfree(ctx, Mprev);
        Mprev = M;
    }
    dfree(ctx, Mprev);
    grow_c(ctx, A, A->k + kb);
    if (kb) {
        ck(ctx, cudaMemcpyAsync(A->c_level + A->k, B->c_level, kb * 4, cudaMemcpyDeviceToDevice, ctx->st), "copy");
        ck(ctx, cudaMemcpyAsync(A->c_rank + A->k, cb_rank, kb * 4, cudaMemcpyDeviceToDevice, ctx->st), "copy");
    }
    A->k += kb;
    dfree(ctx, cb_rank);
    check_device_status(ctx, read_status(ctx));
}

// --------------------------------------------------------------------------
// exp(C[j])
// --------------------------------------------------------------------------

void decompress(lcg_ctx* ctx, const lcg_grammar* G, u32 j, uint8_t* out, u64 cap, uint64_t* out_len, int on_dev) {
    fail_if(ctx, j >= G->k, LCG_EINVAL, "string index out of range");
    u32 lev = 0, r = 0;
    ck(ctx, cudaMemcpyAsync(&lev, G->c_level + j, 4, cudaMemcpyDeviceToHost, ctx->st), "read C");
    ck(ctx, cudaMemcpyAsync(&r, G->c_rank + j, 4, cudaMemcpyDeviceToHost, ctx->st), "read C");
    sync(ctx);
    u32* cur = dalloc<u32>(ctx, 1);
    ck(ctx, cudaMemcpyAsync(cur, &r, 4, cudaMemcpyHostToDevice, ctx->st), "copy");
    u64 cnt = 1;
    for (u32 l = lev; l >= 1; l--) {
        const Level& L = G->lv[l - 1];
        u32* lens = dalloc<u32>(ctx, cnt);
        u64* offs = dalloc<u64>(ctx, cnt);
        ck(ctx, launch_rule_lens(cur, cnt, L.rhs_off, lens, ctx->st), "rule lens");
        u64 grid = 0;
        const u64 stiles = std::max<u64>(1, scan2_tiles_for(cnt));
        ensure_lb(ctx, &ctx->lb2, &ctx->lb2_tiles, stiles, scan2_lb_bytes(stiles));
        ck(ctx, launch_scan2(lens, nullptr, cnt, offs, nullptr, ctx->scratch + 1, ctx->lb2, ++ctx->epoch, ctx->ctr,
                             ctx->ctr_val, ctx->ds, ctx->st, &grid),
           "scan");
        ctx->ctr_val += grid;
        u64 total = 0;
        ck(ctx, cudaMemcpyAsync(&total, ctx->scratch + 1, 8, cudaMemcpyDeviceToHost, ctx->st), "read total");
        check_device_status(ctx, read_status(ctx));
        u32* next = dalloc<u32>(ctx, total);
        ck(ctx, launch_expand(cur, cnt, offs, L.rhs_off, L.rhs, next, ctx->st), "expand");
        ctx->launches += 3;
        dfree(ctx, lens);
        dfree(ctx, offs);
        dfree(ctx, cur);
        cur = next;
        cnt = total;
    }
    *out_len = cnt;
    if (cap < cnt) {
        dfree(ctx, cur);
        sync(ctx);
        fail_if(ctx, true, LCG_EINVAL, "output buffer too small");
    }
    if (on_dev) {
        ck(ctx, launch_to_bytes(cur, cnt, out, ctx->st), "to bytes");
    } else {
        unsigned char* tmp = dalloc<unsigned char>(ctx, cnt);
        ck(ctx, launch_to_bytes(cur, cnt, tmp, ctx->st), "to bytes");
        ck(ctx, cudaMemcpyAsync(out, tmp, cnt, cudaMemcpyDeviceToHost, ctx->st), "copy out");
        dfree(ctx, tmp);
    }
    ctx->launches++;
    dfree(ctx, cur);
    sync(ctx);
}

// --------------------------------------------------------------------------
// exp(C[j]) without allocation: scratch in a static device array
// --------------------------------------------------------------------------
//
// For callers that must not allocate device memory when they expand a string:
// code that runs inside an allocator's or a memory-pressure callback (it
// cannot call back into the allocator), and services that reserve their
// device memory up front and keep no room for transient buffers.  The scratch
// lives in this file-scope array, which every GPU that loads the library
// holds until the process exits.  Host code cannot use the array's name as a
// device address: its address is taken once per device, with that device
// current, by cudaGetSymbolAddress (under a lock, as contexts on several host
// threads may make their first call at once).  Every call shares the array:
// calls that overlap on the GPU race.

constexpr u64 kStaticMaxSymbols = 1ull << 20;  // longest string expanded: 1 MiB
constexpr u64 kStaticLbTiles = 1024;           // look-back slots for one scan of kStaticMaxSymbols

struct StaticScratch {
    u32 cur[kStaticMaxSymbols];
    u32 next[kStaticMaxSymbols];
    u32 lens[kStaticMaxSymbols];
    u64 offs[kStaticMaxSymbols];
    u64 totals[2];
    unsigned char lb[kStaticLbTiles * 48];
};

static __device__ __align__(256) unsigned char g_static_scratch[sizeof(StaticScratch)];

StaticScratch* static_scratch_of_device(lcg_ctx* ctx) {
    static std::mutex mu;
    static StaticScratch* addr[256] = {nullptr};
    fail_if(ctx, ctx->device < 0 || ctx->device >= 256, LCG_EDEVICE, "device index out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[ctx->device]) {
        void* p = nullptr;
        ck(ctx, cudaGetSymbolAddress(&p, g_static_scratch), "cudaGetSymbolAddress");
        addr[ctx->device] = (StaticScratch*)p;
    }
    return addr[ctx->device];
}

void decompress_static(lcg_ctx* ctx, const lcg_grammar* G, u32 j, uint8_t* out, u64 cap, uint64_t* out_len) {
    static_assert(scan2_lb_bytes_static(kStaticLbTiles) <= kStaticLbTiles * 48, "look-back slots");
    fail_if(ctx, j >= G->k, LCG_EINVAL, "string index out of range");
    StaticScratch* sc = static_scratch_of_device(ctx);
    u32 lev = 0, r = 0;
    ck(ctx, cudaMemcpyAsync(&lev, G->c_level + j, 4, cudaMemcpyDeviceToHost, ctx->st), "read C");
    ck(ctx, cudaMemcpyAsync(&r, G->c_rank + j, 4, cudaMemcpyDeviceToHost, ctx->st), "read C");
    sync(ctx);
    u32* cur = sc->cur;
    u32* nxt = sc->next;
    ck(ctx, cudaMemcpyAsync(cur, &r, 4, cudaMemcpyHostToDevice, ctx->st), "copy");
    u64 cnt = 1;
    for (u32 l = lev; l >= 1; l--) {
        const Level& L = G->lv[l - 1];
        ck(ctx, launch_rule_lens(cur, cnt, L.rhs_off, sc->lens, ctx->st), "rule lens");
        // the look-back slots left by an earlier call (any context) must not
        // look published
        ck(ctx, cudaMemsetAsync(sc->lb, 0, sizeof(sc->lb), ctx->st), "clear look-back");
        u64 grid = 0;
        ck(ctx, launch_scan2(sc->lens, nullptr, cnt, sc->offs, nullptr, sc->totals, sc->lb, ++ctx->epoch, ctx->ctr,
                             ctx->ctr_val, ctx->ds, ctx->st, &grid),
           "scan");
        ctx->ctr_val += grid;
        u64 total = 0;
        ck(ctx, cudaMemcpyAsync(&total, sc->totals, 8, cudaMemcpyDeviceToHost, ctx->st), "read total");
        check_device_status(ctx, read_status(ctx));
        if (total > kStaticMaxSymbols) {
            *out_len = total;  // a lower bound of the string's length
            fail_if(ctx, true, LCG_EOVERFLOW,
                    "string longer than the static scratch allows (1048576 symbols); use lcg_decompress");
        }
        ck(ctx, launch_expand(cur, cnt, sc->offs, L.rhs_off, L.rhs, nxt, ctx->st), "expand");
        ctx->launches += 3;
        u32* t = cur;
        cur = nxt;
        nxt = t;
        cnt = total;
    }
    *out_len = cnt;
    fail_if(ctx, cap < cnt, LCG_EINVAL, "output buffer too small");
    ck(ctx, launch_to_bytes(cur, cnt, out, ctx->st), "to bytes");
    ctx->launches++;
    sync(ctx);
}

}  // namespace

// --------------------------------------------------------------------------
// post-processing: RL, then Simp (kernels in post.cu)
// --------------------------------------------------------------------------

struct lcg_pp {
    int device = 0;
    u64 rules = 0, size = 0;
    u32 k = 0;
    u8* kind = nullptr;      // rules
    u64* rhs_off = nullptr;  // rules + 1
    u32* rhs = nullptr;      // size
    u32* c = nullptr;        // k
    lcg_pp_stats stats{};
};

namespace {

void free_pp(lcg_pp* pp) {
    if (!pp) return;
    cudaSetDevice(pp->device);
    cudaFree(pp->kind);
    cudaFree(pp->rhs_off);
    cudaFree(pp->rhs);
    cudaFree(pp->c);
    delete pp;
}

// Exclusive scan of up to two u32 columns (the library's single-pass scan);
// returns the column totals.
void pp_scan(lcg_ctx* ctx, const u32* in0, const u32* in1, u64 n, u64* out0, u64* out1, u64 tot[2]) {
    tot[0] = tot[1] = 0;
    if (n == 0) return;
    u64 grid = 0;
    const u64 stiles = std::max<u64>(1, scan2_tiles_for(n));
    ensure_lb(ctx, &ctx->lb2, &ctx->lb2_tiles, stiles, scan2_lb_bytes(stiles));
    ck(ctx, launch_scan2(in0, in1, n, out0, out1, ctx->scratch + 1, ctx->lb2, ++ctx->epoch, ctx->ctr, ctx->ctr_val,
                         ctx->ds, ctx->st, &grid),
       "scan");
    ctx->ctr_val += grid;
    ctx->launches++;
    ck(ctx, cudaMemcpyAsync(tot, ctx->scratch + 1, 16, cudaMemcpyDeviceToHost, ctx->st), "read totals");
    check_device_status(ctx, read_status(ctx));
}

// Temporary device arrays of one post-processing call, freed in stream order.
struct PPTemps {
    lcg_ctx* ctx;
    std::vector<void*> ptrs;
    template <typename T>
    T* get(u64 n) {
        T* p = dalloc<T>(ctx, n);
        ptrs.push_back(p);
        return p;
    }
    ~PPTemps() {
        for (void* p : ptrs) dfree(ctx, p);
    }
};

void set_u64(lcg_ctx* ctx, u64* dst, u64 v) {
    ck(ctx, cudaMemcpyAsync(dst, &v, 8, cudaMemcpyHostToDevice, ctx->st), "set value");
    sync(ctx);  // v lives on the host stack
}

lcg_pp* postprocess(lcg_ctx* ctx, const lcg_grammar* G) {
    const u32 nl = (u32)G->lv.size();
    fail_if(ctx, nl > (u32)kPPMaxLevels, LCG_EINVAL, "grammar with too many levels");
    if (G->owner && G->owner != ctx) ck(ctx, cudaStreamSynchronize(G->owner->st), "grammar's stream");
    sync(ctx);
    reset_status(ctx);
    PPTemps tmp{ctx, {}};
    PPLevels lv{};
    lv.n = nl;
    std::vector<u32*> uses(nl);
    u64 rl_total = 0, size_before = 0, size_rl = 0;
    // RL, level by level
    for (u32 i = 0; i < nl; i++) {
        const Level& L = G->lv[i];
        const u64 g = L.g;
        size_before += L.G;
        u32* out_len = tmp.get<u32>(g);
        u32* rl_len = tmp.get<u32>(g);
        u64* new_off = tmp.get<u64>(g + 1);
        u64* rl_off = tmp.get<u64>(g);
        ck(ctx, launch_rl_count(L.rhs_off, L.rhs, g, out_len, rl_len, ctx->st), "k_rl_count");
        u64 tot[2];
        pp_scan(ctx, out_len, rl_len, g, new_off, rl_off, tot);
        const u64 Gn = tot[0], R = tot[1];
        set_u64(ctx, new_off + g, Gn);
        u32* new_rhs = tmp.get<u32>(Gn);
        u32* run_y = tmp.get<u32>(R);
        u32* run_len = tmp.get<u32>(R);
        u64* run_pos = tmp.get<u64>(R);
        u64 cap = 64;
        while (cap < 2 * R + 16) cap <<= 1;
        u64* keys = tmp.get<u64>(cap);
        u64* vals = tmp.get<u64>(cap);
        ck(ctx, cudaMemsetAsync(keys, 0xFF, cap * 8, ctx->st), "memset");
        ck(ctx, cudaMemsetAsync(vals, 0xFF, cap * 8, ctx->st), "memset");
        ck(ctx, launch_rl_write(L.rhs_off, L.rhs, g, new_off, rl_off, new_rhs, run_y, run_len, run_pos, keys, vals,
                                cap - 1, ctx->ds, ctx->st),
           "k_rl_write");
        u32* first = tmp.get<u32>(R);
        u64* run_first = tmp.get<u64>(R);
        u64* rank_of = tmp.get<u64>(R);
        ck(ctx, launch_rl_first(run_y, run_len, R, keys, vals, cap - 1, first, run_first, ctx->ds, ctx->st),
           "k_rl_first");
        pp_scan(ctx, first, nullptr, R, rank_of, nullptr, tot);
        const u64 Rd = tot[0];
        u32* rl_y = tmp.get<u32>(Rd);
        u32* rl_l = tmp.get<u32>(Rd);
        ck(ctx, launch_rl_fix(run_y, run_len, run_pos, run_first, rank_of, R, new_rhs, rl_y, rl_l, ctx->ds, ctx->st),
           "k_rl_fix");
        ctx->launches += 4;
        lv.off[i] = new_off;
        lv.rhs[i] = new_rhs;
        lv.g[i] = g;
        lv.nrl[i] = Rd;
        lv.rl_y[i] = rl_y;
        lv.rl_l[i] = rl_l;
        rl_total += Rd;
        size_rl += Gn + 2 * Rd;
        uses[i] = tmp.get<u32>(g);
        lv.pinned[i] = tmp.get<u8>(g);
        ck(ctx, cudaMemsetAsync(uses[i], 0, g * 4, ctx->st), "memset");
        ck(ctx, cudaMemsetAsync(lv.pinned[i], 0, g, ctx->st), "memset");
    }
    // Simp: uses, kept rules, surviving rules and their ids
    for (u32 i = 1; i < nl; i++) {
        ck(ctx, launch_pp_uses(lv.off[i], lv.rhs[i], lv.g[i], uses[i - 1], ctx->st), "k_pp_uses");
        ck(ctx, launch_pp_pin_bases(lv.rl_y[i], lv.nrl[i], lv.pinned[i - 1], ctx->st), "k_pp_pin_bases");
        ctx->launches += 2;
    }
    ck(ctx, launch_pp_pin_roots(G->c_level, G->c_rank, G->k, lv, ctx->st), "k_pp_pin_roots");
    u64 next = 256, removed = 0;
    for (u32 i = 0; i < nl; i++) {
        u32* surv = tmp.get<u32>(lv.g[i]);
        u64* spre = tmp.get<u64>(lv.g[i]);
        ck(ctx, launch_pp_survive(uses[i], lv.pinned[i], lv.g[i], surv, ctx->st), "k_pp_survive");
        u64 tot[2];
        pp_scan(ctx, surv, nullptr, lv.g[i], spre, nullptr, tot);
        lv.surv[i] = surv;
        lv.spre[i] = spre;
        lv.S[i] = tot[0];
        lv.base[i] = next;
        lv.explen[i] = tmp.get<u32>(lv.g[i]);
        lv.dst[i] = tmp.get<u64>(lv.g[i]);
        ck(ctx, cudaMemsetAsync(lv.dst[i], 0xFF, lv.g[i] * 8, ctx->st), "memset");
        next += lv.S[i] + lv.nrl[i];
        removed += lv.g[i] - lv.S[i];
        ctx->launches += 2;
    }
    const u64 rules = next - 256;
    fail_if(ctx, next > 0xffffffffull, LCG_EOVERFLOW, "post-processed grammar with 2^32 symbols or more");
    u32* fin_len = tmp.get<u32>(rules);
    for (u32 i = 0; i < nl; i++) {
        ck(ctx, launch_pp_lengths(lv, i, fin_len, ctx->ds, ctx->st), "k_pp_explen");
        ctx->launches += 2;
    }
    auto* pp = new lcg_pp;
    pp->device = ctx->device;
    pp->rules = rules;
    pp->k = G->k;
    try {
        pp->rhs_off = dalloc<u64>(ctx, rules + 1);
        u64 tot[2];
        pp_scan(ctx, fin_len, nullptr, rules, pp->rhs_off, nullptr, tot);
        pp->size = tot[0];
        set_u64(ctx, pp->rhs_off + rules, pp->size);
        pp->rhs = dalloc<u32>(ctx, pp->size);
        pp->kind = dalloc<u8>(ctx, rules);
        pp->c = dalloc<u32>(ctx, G->k);
        for (u32 i = nl; i-- > 0;) {  // top level first: removed rules learn their place from above
            ck(ctx, launch_pp_write(lv, i, pp->rhs_off, pp->rhs, pp->kind, ctx->ds, ctx->st), "k_pp_place");
            ctx->launches += 2;
        }
        ck(ctx, launch_pp_roots(G->c_level, G->c_rank, G->k, lv, pp->c, ctx->st), "k_pp_roots");
        ctx->launches++;
        check_device_status(ctx, read_status(ctx));
    } catch (...) {
        sync(ctx);
        free_pp(pp);
        throw;
    }
    pp->stats.size_before = size_before;
    pp->stats.size_rl = size_rl;
    pp->stats.size = pp->size;
    pp->stats.rl_rules = rl_total;
    pp->stats.removed = removed;
    pp->stats.rules = rules;
    pp->stats.strings = G->k;
    return pp;
}

}  // namespace

// --------------------------------------------------------------------------
// C entry points
// --------------------------------------------------------------------------

#define LCG_GUARD_BEGIN try {
#define LCG_GUARD_END                                  \
    }                                                  \
    catch (const Fail& f) {                            \
        return f.code;                                 \
    }                                                  \
    catch (const std::bad_alloc&) {                    \
        ctx->err = "host allocation failed";           \
        return LCG_ENOMEM;                             \
    }

extern "C" {

int lcg_ctx_create(int device, const lcg_hash_family* H, void* stream, lcg_ctx** out) {
    if (!out) return LCG_EINVAL;
    *out = nullptr;
    if (!H || H->levels < 2 || H->levels > 4096 || H->m_bits < 1 || H->m_bits > 32 || !H->a || !H->b || !H->c)
        return LCG_EINVAL;
    for (u32 i = 0; i < H->levels; i++)
        if (H->a[i] == 0 || H->a[i] >= kP61 || H->b[i] >= kP61 || H->c[i] == 0 || H->c[i] >= kP61)
            return LCG_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return LCG_EDEVICE;
    lcg_ctx* ctx = new (std::nothrow) lcg_ctx();
    if (!ctx) return LCG_ENOMEM;
    ctx->device = device;
    ctx->a.assign(H->a, H->a + H->levels);
    ctx->b.assign(H->b, H->b + H->levels);
    ctx->c.assign(H->c, H->c + H->levels);
    ctx->levels = H->levels;
    ctx->m_bits = H->m_bits;
    ctx->mmask = (H->m_bits == 32) ? 0xffffffffull : ((1ull << H->m_bits) - 1);
    u64 tag = 1469598103934665603ull;
    for (u32 i = 0; i < H->levels; i++) {
        for (u64 w : {H->a[i], H->b[i], H->c[i]}) tag = (tag ^ w) * 1099511628211ull;
    }
    ctx->tag = (tag ^ ctx->mmask) * 1099511628211ull;
    try {
        ck(ctx, cudaSetDevice(device), "cudaSetDevice");
        ck(ctx, cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device), "device attribute");
        if (ctx->sms < 1) ctx->sms = 1;
        if (stream) {
            ctx->st = (cudaStream_t)stream;
        } else {
            ck(ctx, cudaStreamCreateWithFlags(&ctx->st, cudaStreamNonBlocking), "stream");
            ctx->own_stream = true;
        }
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            u64 thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        ck(ctx, cudaMalloc(&ctx->ds, sizeof(DevStatus)), "cudaMalloc");
        ck(ctx, cudaMalloc(&ctx->rc, sizeof(RoundCounts)), "cudaMalloc");
        ck(ctx, cudaMalloc(&ctx->ctr, sizeof(u64)), "cudaMalloc");
        ck(ctx, cudaMalloc(&ctx->scratch, 8 * sizeof(u64)), "cudaMalloc");
        ck(ctx, cudaMalloc(&ctx->ds_arr, kMaxRounds * sizeof(DevStatus)), "cudaMalloc");
        ck(ctx, cudaMalloc(&ctx->rc_arr, kMaxRounds * sizeof(RoundCounts)), "cudaMalloc");
        ck(ctx, cudaMalloc(&ctx->tot_arr, 3 * kMaxRounds * sizeof(u64)), "cudaMalloc");
        ck(ctx, cudaMemset(ctx->ds, 0, sizeof(DevStatus)), "memset");
        ck(ctx, cudaMemset(ctx->ctr, 0, sizeof(u64)), "memset");
        ck(ctx, cudaMemset(ctx->scratch, 0, 8 * sizeof(u64)), "memset");
        ck(ctx, cudaDeviceSynchronize(), "sync");
    } catch (const Fail& f) {
        lcg_ctx_destroy(ctx);
        return f.code;
    }
    *out = ctx;
    return LCG_OK;
}

void lcg_ctx_destroy(lcg_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    for (lcg_grammar* G : ctx->live) G->owner = nullptr;  // they outlive the context
    ctx->live.clear();
    destroy_graph(ctx);
    if (ctx->upload) cudaFree(ctx->upload);
    for (auto& r : ctx->krecs) {
        if (r.graph) continue;  // destroyed with the graph
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : ctx->evpool) cudaEventDestroy(e);
    if (ctx->lb1) cudaFree(ctx->lb1);
    if (ctx->heads) cudaFree(ctx->heads);
    if (ctx->lb2) cudaFree(ctx->lb2);
    cudaFree(ctx->ds);
    cudaFree(ctx->rc);
    cudaFree(ctx->ctr);
    cudaFree(ctx->scratch);
    cudaFree(ctx->ds_arr);
    cudaFree(ctx->rc_arr);
    cudaFree(ctx->tot_arr);
    if (ctx->own_stream && ctx->st) cudaStreamDestroy(ctx->st);
    delete ctx;
}

const char* lcg_last_error(const lcg_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int lcg_last_build_stats(const lcg_ctx* ctx, lcg_build_stats* out) {
    if (!ctx || !out) return LCG_EINVAL;
    *out = ctx->stats;
    return LCG_OK;
}

int lcg_set_kernel_timing(lcg_ctx* ctx, int enable) {
    if (!ctx || enable < 0 || enable > 2) return LCG_EINVAL;
    ctx->ktime = enable;
    return LCG_OK;
}

int lcg_set_graph(lcg_ctx* ctx, int enable) {
    if (!ctx || enable < 0 || enable > 1) return LCG_EINVAL;
    ctx->use_graph = enable != 0;
    if (!ctx->use_graph) destroy_graph(ctx);
    return LCG_OK;
}

int lcg_set_tuning(lcg_ctx* ctx, const lcg_tuning* t) {
    if (!ctx || !t) return LCG_EINVAL;
    const int maxb = std::max(parse_max_blocks(1), parse_max_blocks(4));
    if (!(t->table_load >= 0.3 && t->table_load <= 0.78) || t->parse_blocks_per_sm > (uint32_t)maxb ||
        t->miss_flush < 32 || t->miss_flush > 256 || (t->table_slots_max != 0 && t->table_slots_max < 1024) ||
        t->tile_stripes < 1 || t->tile_stripes > 16 || !parse_tile_valid(t->parse_tile) ||
        t->parse_tile_min > 1024) {
        ctx->err = "tuning out of range: table_load in [0.3, 0.78], parse_blocks_per_sm <= " + std::to_string(maxb) +
                   ", miss_flush in [32, 256], table_slots_max 0 or >= 1024, tile_stripes in [1, 16], "
                   "parse_tile 1024, 2048 or 4096, parse_tile_min <= 1024";
        return LCG_EINVAL;
    }
    ctx->tuning = *t;
    return LCG_OK;
}

int lcg_get_tuning(const lcg_ctx* ctx, lcg_tuning* t) {
    if (!ctx || !t) return LCG_EINVAL;
    *t = ctx->tuning;
    return LCG_OK;
}

int lcg_last_kernel_times(const lcg_ctx* ctx, lcg_kernel_time* out, uint32_t cap, uint32_t* count) {
    if (!ctx || !count) return LCG_EINVAL;
    *count = (uint32_t)ctx->ktimes.size();
    for (uint32_t x = 0; x < cap && x < ctx->ktimes.size(); x++) out[x] = ctx->ktimes[x];
    return LCG_OK;
}

int lcg_last_kernel_launches(const lcg_ctx* ctx, lcg_kernel_launch* out, uint32_t cap, uint32_t* count) {
    if (!ctx || !count) return LCG_EINVAL;
    *count = (uint32_t)ctx->klaunches.size();
    for (uint32_t x = 0; x < cap && x < ctx->klaunches.size(); x++) out[x] = ctx->klaunches[x];
    return LCG_OK;
}

int lcg_build(lcg_ctx* ctx, const uint8_t* data, const uint64_t* offsets, uint32_t k, int data_on_device,
              lcg_grammar** out) {
    if (!ctx || !out) return LCG_EINVAL;
    const Range range("lcg_build");
    *out = nullptr;
    lcg_grammar* G = nullptr;
    LCG_GUARD_BEGIN
    ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    kt_reset(ctx);
    reset_status(ctx);
    std::vector<uint64_t> shifted;  // offsets into the context's upload buffer
    if (ctx->use_graph && k > 0 && offsets && data && ctx->hint_rounds > 0) {
        std::vector<u64> lens(k);
        bool ok = true;
        for (u32 j = 0; j < k && ok; j++) {
            lens[j] = offsets[j + 1] - offsets[j];
            ok = offsets[j + 1] > offsets[j] && lens[j] >= 2;  // strings of length one: not in graphs
        }
        if (ok && !data_on_device) {
            // host input: into the context's upload buffer, whose address a
            // captured graph can keep; the build then reads it there
            const u64 nbytes = offsets[k] - offsets[0];
            if (ctx->upload_cap < nbytes) {
                if (ctx->upload) {
                    if (ctx->graph) destroy_graph(ctx);
                    dfree(ctx, ctx->upload);
                    ctx->upload = nullptr;
                    ctx->upload_cap = 0;
                }
                const u64 cap = nbytes + nbytes / 8 + 4096;
                ctx->upload = dalloc<unsigned char>(ctx, cap);
                ctx->upload_cap = cap;
            }
            ck(ctx, cudaMemcpyAsync(ctx->upload, data + offsets[0], nbytes, cudaMemcpyHostToDevice, ctx->st),
               "copy input");
            shifted.resize(k + 1);
            for (u32 j = 0; j <= k; j++) shifted[j] = offsets[j] - offsets[0];
            data = ctx->upload;
            offsets = shifted.data();
            data_on_device = 1;
        }
        if (ok) {
            try {
                G = build_with_graph(ctx, data + offsets[0], lens);
            } catch (const Retry&) {
                ctx->plan_slack = std::min(4.0, ctx->plan_slack * 1.6);
                G = nullptr;
                kt_reset(ctx);
                G = new_grammar(ctx);
                build_into(ctx, G, data, offsets, k, data_on_device, false, false);
                ctx->stats.redone = 1;
                ctx->stats.plan_slack = ctx->plan_slack;
                sync(ctx);
                kt_collect(ctx);
                *out = G;
                return LCG_OK;
            }
            if (G) {
                ctx->plan_slack = std::max(1.0, ctx->plan_slack * 0.97);
                ctx->stats.plan_slack = ctx->plan_slack;
                kt_collect(ctx);
                *out = G;
                return LCG_OK;
            }
        }
    }
    G = new_grammar(ctx);
    try {
        build_into(ctx, G, data, offsets, k, data_on_device, false, true);
        if (ctx->stats.async_rounds > 0) ctx->plan_slack = std::max(1.0, ctx->plan_slack * 0.97);
    } catch (const Retry&) {
        ctx->plan_slack = std::min(4.0, ctx->plan_slack * 1.6);
        // the rounds planned from the previous build did not fit: round by round
        sync(ctx);
        free_grammar_now(G);
        G = nullptr;
        kt_reset(ctx);
        G = new_grammar(ctx);
        build_into(ctx, G, data, offsets, k, data_on_device, false, false);
        ctx->stats.redone = 1;
    }
    ctx->stats.plan_slack = ctx->plan_slack;
    sync(ctx);
    kt_collect(ctx);
    *out = G;
    return LCG_OK;
    }
    catch (const Fail& f) {
        cudaStreamSynchronize(ctx->st);
        free_grammar_now(G);
        return f.code;
    }
    catch (const std::bad_alloc&) {
        ctx->err = "host allocation failed";
        cudaStreamSynchronize(ctx->st);
        free_grammar_now(G);
        return LCG_ENOMEM;
    }
}

int lcg_build_into(lcg_ctx* ctx, lcg_grammar* resident, const uint8_t* data, const uint64_t* offsets, uint32_t k,
                   int data_on_device) {
    if (!ctx || !resident) return LCG_EINVAL;
    const Range range("lcg_build_into");
    if (resident->tag != ctx->tag) {
        ctx->err = "resident grammar of another hash family";
        return LCG_EMISMATCH;
    }
    LCG_GUARD_BEGIN
    ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    kt_reset(ctx);
    reset_status(ctx);
    build_into(ctx, resident, data, offsets, k, data_on_device, true, false);
    sync(ctx);
    kt_collect(ctx);
    return LCG_OK;
    LCG_GUARD_END
}

int lcg_merge(lcg_ctx* ctx, lcg_grammar* a, const lcg_grammar* b) {
    if (!ctx || !a || !b) return LCG_EINVAL;
    const Range range("lcg_merge");
    LCG_GUARD_BEGIN
    ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    kt_reset(ctx);
    reset_status(ctx);
    merge(ctx, a, b);
    kt_collect(ctx);
    return LCG_OK;
    LCG_GUARD_END
}

int lcg_decompress(lcg_ctx* ctx, const lcg_grammar* G, uint32_t j, uint8_t* out, uint64_t cap, uint64_t* out_len,
                   int out_on_device) {
    if (!ctx || !G || !out_len) return LCG_EINVAL;
    const Range range("lcg_decompress");
    LCG_GUARD_BEGIN
    ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    decompress(ctx, G, j, out, cap, out_len, out_on_device);
    return LCG_OK;
    LCG_GUARD_END
}

int lcg_decompress_static(lcg_ctx* ctx, const lcg_grammar* G, uint32_t j, uint8_t* out_dev, uint64_t cap,
                          uint64_t* out_len) {
    if (!ctx || !G || !out_dev || !out_len) return LCG_EINVAL;
    LCG_GUARD_BEGIN
    ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    decompress_static(ctx, G, j, out_dev, cap, out_len);
    return LCG_OK;
    LCG_GUARD_END
}

int lcg_selftest_wait_timeout(lcg_ctx* ctx) {
    if (!ctx) return LCG_EINVAL;
    LCG_GUARD_BEGIN
    ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    kt_reset(ctx);
    reset_status(ctx);
    // A scan of 8 tiles whose tile counter is read one ahead: the first block
    // takes tile 1 and waits for a tile 0 that no block takes.  Every block
    // stays in bounds (tiles 1..8 of the 8 look-back slots sized below; tile 8
    // returns at once), and the wait ends with kErrTimeout.
    const u64 n = 16384;  // 8 tiles of the scan
    const u64 tiles = scan2_tiles_for(n);
    ensure_lb(ctx, &ctx->lb2, &ctx->lb2_tiles, tiles + 1, scan2_lb_bytes(tiles + 1));
    u32* in = dalloc<u32>(ctx, n);
    u64* out = dalloc<u64>(ctx, n);
    ck(ctx, cudaMemsetAsync(in, 0, n * sizeof(u32), ctx->st), "memset");
    ck(ctx, cudaMemsetAsync(ctx->ds, 0, sizeof(DevStatus), ctx->st), "reset status");
    u64 grid = 0;
    ck(ctx, launch_scan2(in, nullptr, n, out, nullptr, ctx->scratch + 1, ctx->lb2, ++ctx->epoch, ctx->ctr,
                         ctx->ctr_val - 1, ctx->ds, ctx->st, &grid, nullptr),
       "scan");
    ctx->ctr_val += grid;
    dfree(ctx, in);
    dfree(ctx, out);
    const DevStatus st = read_status(ctx);
    check_device_status(ctx, st);
    return LCG_OK;
    LCG_GUARD_END
}

int lcg_grammar_shape(const lcg_grammar* G, uint32_t* k, uint32_t* nlevels) {
    if (!G) return LCG_EINVAL;
    if (k) *k = G->k;
    if (nlevels) *nlevels = (uint32_t)G->lv.size();
    return LCG_OK;
}

int lcg_level_size(const lcg_grammar* G, uint32_t level, uint64_t* g, uint64_t* Gsz) {
    if (!G || level < 1 || level > G->lv.size()) return LCG_EINVAL;
    if (g) *g = G->lv[level - 1].g;
    if (Gsz) *Gsz = G->lv[level - 1].G;
    return LCG_OK;
}

int lcg_export_level(lcg_ctx* ctx, const lcg_grammar* G, uint32_t level, uint64_t* rhs_off, uint32_t* rhs,
                     uint32_t* F) {
    if (!ctx || !G || level < 1 || level > G->lv.size()) return LCG_EINVAL;
    LCG_GUARD_BEGIN
    ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    const Level& L = G->lv[level - 1];
    if (rhs_off)
        ck(ctx, cudaMemcpyAsync(rhs_off, L.rhs_off, (L.g + 1) * 8, cudaMemcpyDeviceToHost, ctx->st), "export");
    if (rhs && L.G) ck(ctx, cudaMemcpyAsync(rhs, L.rhs, L.G * 4, cudaMemcpyDeviceToHost, ctx->st), "export");
    if (F && L.g) ck(ctx, cudaMemcpyAsync(F, L.F, L.g * 4, cudaMemcpyDeviceToHost, ctx->st), "export");
    sync(ctx);
    return LCG_OK;
    LCG_GUARD_END
}

int lcg_export_start(lcg_ctx* ctx, const lcg_grammar* G, uint32_t* F0, uint32_t* c_level, uint32_t* c_rank) {
    if (!ctx || !G) return LCG_EINVAL;
    LCG_GUARD_BEGIN
    ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    if (F0) ck(ctx, cudaMemcpyAsync(F0, G->F0, 256 * 4, cudaMemcpyDeviceToHost, ctx->st), "export");
    if (c_level && G->k)
        ck(ctx, cudaMemcpyAsync(c_level, G->c_level, G->k * 4, cudaMemcpyDeviceToHost, ctx->st), "export");
    if (c_rank && G->k)
        ck(ctx, cudaMemcpyAsync(c_rank, G->c_rank, G->k * 4, cudaMemcpyDeviceToHost, ctx->st), "export");
    sync(ctx);
    return LCG_OK;
    LCG_GUARD_END
}

int lcg_import(lcg_ctx* ctx, uint32_t k, uint32_t nlevels, const uint64_t* g, const uint64_t* const* rhs_off,
               const uint32_t* const* rhs, const uint32_t* const* F, const uint32_t* c_level, const uint32_t* c_rank,
               lcg_grammar** out) {
    if (!ctx || !out) return LCG_EINVAL;
    *out = nullptr;
    if (nlevels && (!g || !rhs_off || !rhs || !F)) return LCG_EINVAL;
    if (k && (!c_level || !c_rank)) return LCG_EINVAL;
    lcg_grammar* G = nullptr;
    try {
        ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
        kt_reset(ctx);
        fail_if(ctx, nlevels >= ctx->levels, LCG_ELEVELS, "grammar has more levels than the hash family has functions");
        // host checks: offsets, symbol ranges and C entries name existing rules
        for (u32 i = 1; i <= nlevels; i++) {
            const u64 gi = g[i - 1];
            fail_if(ctx, gi > kMaxRank, LCG_EOVERFLOW, "level with 2^31 rules or more");
            fail_if(ctx, rhs_off[i - 1] == nullptr || (gi && (rhs[i - 1] == nullptr || F[i - 1] == nullptr)),
                    LCG_EINVAL, "missing array of level " + std::to_string(i));
            const uint64_t* ro = rhs_off[i - 1];
            fail_if(ctx, ro[0] != 0, LCG_EINVAL, "rhs_off of level " + std::to_string(i) + " does not start at 0");
            for (u64 r = 0; r < gi; r++)
                fail_if(ctx, ro[r + 1] <= ro[r], LCG_EINVAL,
                        "rule " + std::to_string(r) + " of level " + std::to_string(i) + " is empty or misplaced");
            const u64 prev = (i == 1) ? 256 : g[i - 2];
            const uint32_t* x = rhs[i - 1];
            for (u64 y = 0; y < ro[gi]; y++)
                fail_if(ctx, x[y] >= prev, LCG_EINVAL,
                        "level " + std::to_string(i) + " names a symbol outside level " + std::to_string(i - 1));
        }
        for (u32 j = 0; j < k; j++) {
            const u32 lvl = c_level[j];
            fail_if(ctx, lvl > nlevels, LCG_EINVAL, "C entry " + std::to_string(j) + " names a missing level");
            const u64 lim = (lvl == 0) ? 256 : g[lvl - 1];
            fail_if(ctx, c_rank[j] >= lim, LCG_EINVAL, "C entry " + std::to_string(j) + " names a missing rule");
        }
        reset_status(ctx);
        G = new_grammar(ctx);
        if (k) {
            grow_c(ctx, G, k);
            ck(ctx, cudaMemcpyAsync(G->c_level, c_level, (u64)k * 4, cudaMemcpyHostToDevice, ctx->st), "import");
            ck(ctx, cudaMemcpyAsync(G->c_rank, c_rank, (u64)k * 4, cudaMemcpyHostToDevice, ctx->st), "import");
            G->k = k;
        }
        for (u32 i = 1; i <= nlevels; i++) {
            const u64 gi = g[i - 1], Gi = rhs_off[i - 1][gi];
            G->lv.emplace_back();
            Level& L = G->lv.back();
            grow_level(ctx, L, gi, Gi);
            ck(ctx, cudaMemcpyAsync(L.rhs_off, rhs_off[i - 1], (gi + 1) * 8, cudaMemcpyHostToDevice, ctx->st), "import");
            if (Gi) ck(ctx, cudaMemcpyAsync(L.rhs, rhs[i - 1], Gi * 4, cudaMemcpyHostToDevice, ctx->st), "import");
            if (gi) ck(ctx, cudaMemcpyAsync(L.F, F[i - 1], gi * 4, cudaMemcpyHostToDevice, ctx->st), "import");
            L.g = gi;
            L.G = Gi;
            L.rvalid = false;
            ck(ctx, launch_check_fp(L.rhs, L.rhs_off, gi, fprev_of(G, i), level_hash(ctx, i), L.F, ctx->ds, ctx->st),
               "k_check_fp");
            ctx->launches++;
        }
        const DevStatus st = read_status(ctx);
        fail_if(ctx, st.error == kErrMismatch, LCG_EMISMATCH,
                "imported fingerprints differ from those of this context's hash family");
        check_device_status(ctx, st);
        *out = G;
        return LCG_OK;
    } catch (const Fail& f) {
        cudaStreamSynchronize(ctx->st);
        free_grammar_now(G);
        return f.code;
    } catch (const std::bad_alloc&) {
        ctx->err = "host allocation failed";
        cudaStreamSynchronize(ctx->st);
        free_grammar_now(G);
        return LCG_ENOMEM;
    }
}

int lcg_string_roots(lcg_ctx* ctx, const lcg_grammar* G, uint32_t j0, uint32_t count, uint32_t* level,
                     uint32_t* rank, uint32_t* fp) {
    if (!ctx || !G || (count && (!level || !rank || !fp))) return LCG_EINVAL;
    if ((u64)j0 + count > G->k) {
        ctx->err = "string index out of range";
        return LCG_EINVAL;
    }
    if (count == 0) return LCG_OK;
    LCG_GUARD_BEGIN
    ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    fail_if(ctx, G->lv.size() > 64, LCG_ELEVELS, "grammar with more than 64 levels");
    FTable ft{};
    ft.F[0] = G->F0;
    for (u32 i = 1; i <= G->lv.size(); i++) ft.F[i] = G->lv[i - 1].F;
    ft.n = (u32)G->lv.size() + 1;
    u32* d = dalloc<u32>(ctx, 3ull * count);
    ck(ctx, launch_roots(G->c_level, G->c_rank, j0, count, ft, d, ctx->st), "k_roots");
    std::vector<u32> h(3ull * count);
    ck(ctx, cudaMemcpyAsync(h.data(), d, h.size() * 4, cudaMemcpyDeviceToHost, ctx->st), "roots");
    dfree(ctx, d);
    sync(ctx);
    for (u32 x = 0; x < count; x++) {
        level[x] = h[3 * x];
        rank[x] = h[3 * x + 1];
        fp[x] = h[3 * x + 2];
    }
    return LCG_OK;
    LCG_GUARD_END
}

// ---- packed form: one buffer, every section 8-byte aligned ----------------

constexpr u64 kPackMagic = 0x4C434753ull;  // "LCGS"

static u64 pad8(u64 b) { return (b + 7) & ~7ull; }

static u64 packed_bytes(const lcg_grammar* G) {
    const u64 nl = G->lv.size();
    u64 b = 8 * (3 + 2 * nl);
    for (const Level& L : G->lv) b += 8 * (L.g + 1) + pad8(4 * L.G) + pad8(4 * L.g);
    return b + 2 * pad8(4ull * G->k) + 4 * 256;
}

int lcg_packed_size(const lcg_grammar* G, uint64_t* bytes) {
    if (!G || !bytes) return LCG_EINVAL;
    *bytes = packed_bytes(G);
    return LCG_OK;
}

int lcg_export_packed(lcg_ctx* ctx, const lcg_grammar* G, void* out, uint64_t cap) {
    if (!ctx || !G || !out) return LCG_EINVAL;
    LCG_GUARD_BEGIN
    ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    fail_if(ctx, ((uintptr_t)out & 7) != 0, LCG_EINVAL, "packed buffer must be 8-byte aligned");
    fail_if(ctx, cap < packed_bytes(G), LCG_EINVAL, "packed buffer too small");
    unsigned char* o = (unsigned char*)out;
    u64* head = (u64*)o;
    const u64 nl = G->lv.size();
    head[0] = kPackMagic;
    head[1] = G->k;
    head[2] = nl;
    for (u64 i = 0; i < nl; i++) {
        head[3 + 2 * i] = G->lv[i].g;
        head[4 + 2 * i] = G->lv[i].G;
    }
    u64 pos = 8 * (3 + 2 * nl);
    auto d2h = [&](const void* src, u64 bytes, u64 span) {
        if (bytes) ck(ctx, cudaMemcpyAsync(o + pos, src, bytes, cudaMemcpyDeviceToHost, ctx->st), "export");
        if (span > bytes) std::memset(o + pos + bytes, 0, span - bytes);
        pos += span;
    };
    for (const Level& L : G->lv) {
        d2h(L.rhs_off, 8 * (L.g + 1), 8 * (L.g + 1));
        d2h(L.rhs, 4 * L.G, pad8(4 * L.G));
        d2h(L.F, 4 * L.g, pad8(4 * L.g));
    }
    d2h(G->c_level, 4ull * G->k, pad8(4ull * G->k));
    d2h(G->c_rank, 4ull * G->k, pad8(4ull * G->k));
    d2h(G->F0, 4 * 256, 4 * 256);
    sync(ctx);
    return LCG_OK;
    LCG_GUARD_END
}

int lcg_import_packed(lcg_ctx* ctx, const void* buf, uint64_t size, lcg_grammar** out) {
    if (!ctx || !buf || !out) return LCG_EINVAL;
    *out = nullptr;
    auto bad = [&](const char* why) {
        ctx->err = std::string("packed grammar: ") + why;
        return LCG_EINVAL;
    };
    if (((uintptr_t)buf & 7) != 0) return bad("buffer must be 8-byte aligned");
    const unsigned char* b = (const unsigned char*)buf;
    const u64* head = (const u64*)b;
    if (size < 24 || head[0] != kPackMagic) return bad("not a packed grammar");
    const u64 k = head[1], nl = head[2];
    if (k > 0xffffffffull || nl > 4096 || size < 8 * (3 + 2 * nl)) return bad("malformed header");
    std::vector<uint64_t> g(nl), Gs(nl);
    std::vector<const uint64_t*> ro(nl);
    std::vector<const uint32_t*> rhs(nl), F(nl);
    u64 pos = 8 * (3 + 2 * nl);
    for (u64 i = 0; i < nl; i++) {
        g[i] = head[3 + 2 * i];
        Gs[i] = head[4 + 2 * i];
        if (g[i] > kMaxRank || Gs[i] > (1ull << 40)) return bad("malformed level sizes");
        const u64 need = 8 * (g[i] + 1) + pad8(4 * Gs[i]) + pad8(4 * g[i]);
        if (pos + need > size) return bad("truncated");
        ro[i] = (const uint64_t*)(b + pos);
        rhs[i] = (const uint32_t*)(b + pos + 8 * (g[i] + 1));
        F[i] = (const uint32_t*)(b + pos + 8 * (g[i] + 1) + pad8(4 * Gs[i]));
        if (ro[i][g[i]] != Gs[i]) return bad("level sizes disagree with the offsets");
        pos += need;
    }
    if (pos + 2 * pad8(4 * k) + 4 * 256 != size) return bad("wrong size");
    const uint32_t* cl = (const uint32_t*)(b + pos);
    const uint32_t* cr = (const uint32_t*)(b + pos + pad8(4 * k));
    const uint32_t* F0 = (const uint32_t*)(b + pos + 2 * pad8(4 * k));
    lcg_grammar* G = nullptr;
    const int rc = lcg_import(ctx, (uint32_t)k, (uint32_t)nl, g.data(), ro.data(), rhs.data(), F.data(), cl, cr, &G);
    if (rc != LCG_OK) return rc;
    // F^0 must be the context's too
    uint32_t mine[256];
    if (cudaMemcpyAsync(mine, G->F0, sizeof(mine), cudaMemcpyDeviceToHost, ctx->st) != cudaSuccess ||
        cudaStreamSynchronize(ctx->st) != cudaSuccess) {
        free_grammar_now(G);
        ctx->err = "read F0";
        return LCG_EDEVICE;
    }
    if (std::memcmp(mine, F0, sizeof(mine)) != 0) {
        free_grammar_now(G);
        ctx->err = "packed grammar: F0 of another hash family";
        return LCG_EMISMATCH;
    }
    *out = G;
    return LCG_OK;
}

// ---- VByte form (Sec. 4, resource usage) ---------------------------------

constexpr u64 kVbMagic = 0x4C434756ull;  // "LCGV"

static int sm_count(lcg_ctx* ctx) {
    int sms = 0;
    ck(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device), "device attribute");
    return sms > 0 ? sms : 1;
}

// Exclusive scan of `cnt` (u32) into `off` (u64); the sum goes to totals[0].
static void vb_scan(lcg_ctx* ctx, const u32* cnt, u64 tiles, u64* off, u64* totals) {
    if (tiles == 0) return;
    u64 grid = 0;
    const u64 stiles = std::max<u64>(1, scan2_tiles_for(tiles));
    ensure_lb(ctx, &ctx->lb2, &ctx->lb2_tiles, stiles, scan2_lb_bytes(stiles));
    const int h = kt_begin(ctx, "k_scan2", 12.0 * (double)tiles);
    ck(ctx, launch_scan2(cnt, nullptr, tiles, off, nullptr, totals, ctx->lb2, ++ctx->epoch, ctx->ctr, ctx->ctr_val,
                         ctx->ds, ctx->st, &grid),
       "scan");
    kt_end(ctx, h);
    ctx->ctr_val += grid;
    ctx->launches++;
}

// Encode step 1: stream bytes per tile of one column (the u32 array `vals`,
// or the rule lengths of `offs`), scanned into tile offsets; the column's
// stream length goes to totals[0] (device).
static void vb_count_col(lcg_ctx* ctx, const u32* vals, const u64* offs, u64 n, u32* tile_bytes, u64* tile_off,
                         u64* totals) {
    const u64 tiles = vb_encode_tiles(n);
    if (tiles == 0) return;
    const int h = kt_begin(ctx, "k_vb_tile_bytes", (offs ? 8.0 : 4.0) * (double)n);
    ck(ctx, launch_vb_tile_bytes(vals, offs, n, tile_bytes, ctx->st), "k_vb_tile_bytes");
    kt_end(ctx, h);
    ctx->launches++;
    vb_scan(ctx, tile_bytes, tiles, tile_off, totals);
}

// Encode step 2: the column's stream at dst (nb bytes in all).
static void vb_write_col(lcg_ctx* ctx, const u32* vals, const u64* offs, u64 n, const u64* tile_off, u8* dst, bool pad,
                         u64 nb) {
    if (n == 0) return;
    const int h = kt_begin(ctx, "k_vb_write", (offs ? 8.0 : 4.0) * (double)n + (double)nb);
    ck(ctx, launch_vb_write(vals, offs, n, tile_off, dst, pad, ctx->st), "k_vb_write");
    kt_end(ctx, h);
    ctx->launches++;
}

// Scratch of the decode of one column: tile counts and offsets.
struct VbTemps {
    u32* cnt = nullptr;
    u64* off = nullptr;
};

// Decode nb bytes into exactly n values in [lo, hi) at vals.
static void vb_decode_col(lcg_ctx* ctx, const u8* src, u64 nb, u64 n, u64 lo, u64 hi, u32* vals, const VbTemps& t,
                          u64* totals) {
    const u64 tiles = vb_decode_tiles(nb);
    if (tiles == 0) return;
    int h = kt_begin(ctx, "k_vb_tile_ends", (double)nb);
    ck(ctx, launch_vb_tile_ends(src, nb, t.cnt, ctx->st), "k_vb_tile_ends");
    kt_end(ctx, h);
    ctx->launches++;
    vb_scan(ctx, t.cnt, tiles, t.off, totals);
    h = kt_begin(ctx, "k_vb_dwrite", (double)nb + 4.0 * (double)n);
    ck(ctx, launch_vb_dwrite(src, nb, n, lo, hi, t.off, vals, ctx->ds, ctx->st), "k_vb_dwrite");
    kt_end(ctx, h);
    ctx->launches++;
}

// Bytes of each level's two VByte streams: [2 i] rule lengths, [2 i + 1]
// right-hand sides of level i + 1.
static std::vector<u64> vb_section_bytes(lcg_ctx* ctx, const lcg_grammar* G) {
    const u64 nl = G->lv.size();
    std::vector<u64> nb(2 * nl, 0);
    if (nl == 0) return nb;
    u64* d = dalloc<u64>(ctx, 2 * nl);
    ck(ctx, cudaMemsetAsync(d, 0, 16 * nl, ctx->st), "memset");
    const int sms = sm_count(ctx);
    for (u64 i = 0; i < nl; i++) {
        const Level& L = G->lv[i];
        ck(ctx, launch_vb_count(nullptr, L.rhs_off, L.g, d + 2 * i, sms, ctx->st), "k_vb_count");
        ck(ctx, launch_vb_count(L.rhs, nullptr, L.G, d + 2 * i + 1, sms, ctx->st), "k_vb_count");
        ctx->launches += (L.g != 0) + (L.G != 0);
    }
    ck(ctx, cudaMemcpyAsync(nb.data(), d, 16 * nl, cudaMemcpyDeviceToHost, ctx->st), "read sizes");
    dfree(ctx, d);
    sync(ctx);
    return nb;
}

static u64 vb_total_bytes(const lcg_grammar* G, const std::vector<u64>& nb) {
    const u64 nl = G->lv.size();
    u64 b = 24 + 32 * nl;
    for (u64 i = 0; i < nl; i++) b += pad8(nb[2 * i]) + pad8(nb[2 * i + 1]) + pad8(4 * G->lv[i].g);
    return b + 2 * pad8(4ull * G->k) + 4 * 256;
}

int lcg_vbyte_encode(lcg_ctx* ctx, const uint32_t* in, uint64_t n, uint8_t* out, uint64_t cap, uint64_t* out_bytes) {
    if (!ctx || !out_bytes || (n && (!in || !out))) return LCG_EINVAL;
    const Range range("lcg_vbyte_encode");
    u32* cnt = nullptr;
    u64* off = nullptr;
    try {
        ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
        kt_reset(ctx);
        reset_status(ctx);
        *out_bytes = 0;
        if (n == 0) return LCG_OK;
        const u64 tiles = vb_encode_tiles(n);
        cnt = dalloc<u32>(ctx, tiles);
        off = dalloc<u64>(ctx, tiles);
        vb_count_col(ctx, in, nullptr, n, cnt, off, ctx->scratch + 1);
        u64 nb = 0;
        ck(ctx, cudaMemcpyAsync(&nb, ctx->scratch + 1, 8, cudaMemcpyDeviceToHost, ctx->st), "read size");
        sync(ctx);
        *out_bytes = nb;
        fail_if(ctx, cap < nb, LCG_EINVAL, "output buffer too small");
        vb_write_col(ctx, in, nullptr, n, off, out, false, nb);
        dfree(ctx, cnt);
        dfree(ctx, off);
        cnt = nullptr;
        off = nullptr;
        const DevStatus st = read_status(ctx);
        kt_collect(ctx);
        check_device_status(ctx, st);
        return LCG_OK;
    } catch (const Fail& f) {
        cudaStreamSynchronize(ctx->st);
        if (cnt) cudaFree(cnt);
        if (off) cudaFree(off);
        return f.code;
    }
}

int lcg_vbyte_decode(lcg_ctx* ctx, const uint8_t* in, uint64_t nbytes, uint32_t* out, uint64_t n) {
    if (!ctx || (nbytes && !in) || (n && !out)) return LCG_EINVAL;
    const Range range("lcg_vbyte_decode");
    VbTemps t;
    try {
        ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
        kt_reset(ctx);
        fail_if(ctx, nbytes < n || nbytes > 5 * n, LCG_EINVAL, "stream length does not fit the value count");
        if (n == 0) return LCG_OK;
        reset_status(ctx);
        const u64 tiles = vb_decode_tiles(nbytes);
        t.cnt = dalloc<u32>(ctx, tiles);
        t.off = dalloc<u64>(ctx, tiles);
        vb_decode_col(ctx, in, nbytes, n, 0, 1ull << 32, out, t, ctx->scratch + 1);
        dfree(ctx, t.cnt);
        dfree(ctx, t.off);
        t = VbTemps{};
        const DevStatus st = read_status(ctx);
        kt_collect(ctx);
        check_device_status(ctx, st);
        return LCG_OK;
    } catch (const Fail& f) {
        cudaStreamSynchronize(ctx->st);
        if (t.cnt) cudaFree(t.cnt);
        if (t.off) cudaFree(t.off);
        return f.code;
    }
}

int lcg_vbyte_size(lcg_ctx* ctx, const lcg_grammar* G, uint64_t* bytes) {
    if (!ctx || !G || !bytes) return LCG_EINVAL;
    LCG_GUARD_BEGIN
    ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    fail_if(ctx, G->device != ctx->device, LCG_EINVAL, "grammar on another device");
    *bytes = vb_total_bytes(G, vb_section_bytes(ctx, G));
    return LCG_OK;
    LCG_GUARD_END
}

int lcg_export_vbyte(lcg_ctx* ctx, const lcg_grammar* G, void* out, uint64_t cap, int out_on_device,
                     uint64_t* bytes) {
    if (!ctx || !G || !out) return LCG_EINVAL;
    const Range range("lcg_export_vbyte");
    std::vector<void*> temps;
    try {
        ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
        fail_if(ctx, G->device != ctx->device, LCG_EINVAL, "grammar on another device");
        fail_if(ctx, ((uintptr_t)out & 7) != 0, LCG_EINVAL, "VByte buffer must be 8-byte aligned");
        kt_reset(ctx);
        reset_status(ctx);
        const u64 nl = G->lv.size();
        // columns: [2 i] rule lengths, [2 i + 1] right-hand sides of level i + 1;
        // one launch per step over all of them
        const u32 ncols = (u32)(2 * nl);
        fail_if(ctx, ncols > (u32)kVbMaxCols, LCG_EINVAL, "too many levels");
        std::vector<VbEncCol> cols(ncols + 1, VbEncCol{nullptr, nullptr, 0, 0, nullptr});
        u64 T = 0;
        for (u32 c = 0; c < ncols; c++) {
            const Level& L = G->lv[c / 2];
            cols[c] = (c % 2) ? VbEncCol{L.rhs, nullptr, L.G, T, nullptr} : VbEncCol{nullptr, L.rhs_off, L.g, T, nullptr};
            T += vb_encode_tiles(cols[c].n);
        }
        cols[ncols].tile0 = T;
        double in_bytes = 0, out_bytes = 0;
        for (u32 c = 0; c < ncols; c++) in_bytes += (c % 2 ? 4.0 : 8.0) * (double)cols[c].n;
        VbEncCol* dcols = dalloc<VbEncCol>(ctx, ncols + 1);
        temps.push_back(dcols);
        u32* cnt = dalloc<u32>(ctx, T);
        temps.push_back(cnt);
        u64* off = dalloc<u64>(ctx, T);
        temps.push_back(off);
        u64* colb = dalloc<u64>(ctx, ncols + 1);
        temps.push_back(colb);
        ck(ctx, cudaMemsetAsync(colb, 0, 8 * (ncols + 1), ctx->st), "memset");
        ck(ctx, cudaMemcpyAsync(dcols, cols.data(), sizeof(VbEncCol) * (ncols + 1), cudaMemcpyHostToDevice, ctx->st),
           "columns");
        if (T) {
            const int h = kt_begin(ctx, "k_vb_tile_bytes", in_bytes);
            ck(ctx, launch_vb_tile_bytes_all(dcols, ncols, T, cnt, colb, ctx->st), "k_vb_tile_bytes");
            kt_end(ctx, h);
            ctx->launches++;
            vb_scan(ctx, cnt, T, off, ctx->scratch + 1);
        }
        std::vector<u64> nb(ncols + 1);
        ck(ctx, cudaMemcpyAsync(nb.data(), colb, 8 * (ncols + 1), cudaMemcpyDeviceToHost, ctx->st), "read sizes");
        sync(ctx);
        for (u32 c = 0; c < ncols; c++) out_bytes += (double)nb[c];
        const u64 total = vb_total_bytes(G, nb);
        if (bytes) *bytes = total;
        fail_if(ctx, cap < total, LCG_EINVAL, "VByte buffer too small");
        u8* dst = (u8*)out;
        if (!out_on_device) {
            dst = dalloc<u8>(ctx, total);
            temps.push_back(dst);
        }
        std::vector<u64> head(3 + 4 * nl);
        head[0] = kVbMagic;
        head[1] = G->k;
        head[2] = nl;
        for (u64 i = 0; i < nl; i++) {
            head[3 + 4 * i] = G->lv[i].g;
            head[4 + 4 * i] = G->lv[i].G;
            head[5 + 4 * i] = nb[2 * i];
            head[6 + 4 * i] = nb[2 * i + 1];
        }
        ck(ctx, cudaMemcpyAsync(dst, head.data(), 8 * head.size(), cudaMemcpyHostToDevice, ctx->st), "header");
        u64 pos = 8 * head.size();
        auto copy_u32 = [&](const u32* src, u64 n) {
            if (n) ck(ctx, cudaMemcpyAsync(dst + pos, src, 4 * n, cudaMemcpyDeviceToDevice, ctx->st), "copy");
            if ((4 * n) & 7) ck(ctx, cudaMemsetAsync(dst + pos + 4 * n, 0, 4, ctx->st), "pad");
            pos += pad8(4 * n);
        };
        for (u64 i = 0; i < nl; i++) {
            const Level& L = G->lv[i];
            cols[2 * i].dst = dst + pos;
            pos += pad8(nb[2 * i]);
            cols[2 * i + 1].dst = dst + pos;
            pos += pad8(nb[2 * i + 1]);
            copy_u32(L.F, L.g);
        }
        if (T) {
            ck(ctx, cudaMemcpyAsync(dcols, cols.data(), sizeof(VbEncCol) * (ncols + 1), cudaMemcpyHostToDevice,
                                    ctx->st),
               "columns");
            const int h = kt_begin(ctx, "k_vb_write", in_bytes + out_bytes);
            ck(ctx, launch_vb_write_all(dcols, ncols, T, off, ctx->st), "k_vb_write");
            kt_end(ctx, h);
            ctx->launches++;
        }
        copy_u32(G->c_level, G->k);
        copy_u32(G->c_rank, G->k);
        copy_u32(G->F0, 256);
        fail_if(ctx, pos != total, LCG_EDEVICE, "VByte layout");
        if (!out_on_device) ck(ctx, cudaMemcpyAsync(out, dst, total, cudaMemcpyDeviceToHost, ctx->st), "export");
        for (void* p : temps) dfree(ctx, p);
        temps.clear();
        const DevStatus st = read_status(ctx);
        kt_collect(ctx);
        check_device_status(ctx, st);
        return LCG_OK;
    } catch (const Fail& f) {
        cudaStreamSynchronize(ctx->st);
        for (void* p : temps) cudaFree(p);
        return f.code;
    } catch (const std::bad_alloc&) {
        ctx->err = "host allocation failed";
        cudaStreamSynchronize(ctx->st);
        for (void* p : temps) cudaFree(p);
        return LCG_ENOMEM;
    }
}

int lcg_import_vbyte(lcg_ctx* ctx, const void* buf, uint64_t size, int buf_on_device, lcg_grammar** out) {
    if (!ctx || !buf || !out) return LCG_EINVAL;
    *out = nullptr;
    const Range range("lcg_import_vbyte");
    lcg_grammar* G = nullptr;
    u8* staging = nullptr;
    std::vector<void*> temps;
    try {
        ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
        kt_reset(ctx);
        fail_if(ctx, ((uintptr_t)buf & 7) != 0, LCG_EINVAL, "VByte buffer must be 8-byte aligned");
        fail_if(ctx, size < 24, LCG_EINVAL, "not a VByte grammar");
        const u8* b = (const u8*)buf;
        auto read_host = [&](void* dst, u64 off, u64 n) {
            if (n == 0) return;
            if (buf_on_device) {
                ck(ctx, cudaMemcpyAsync(dst, b + off, n, cudaMemcpyDeviceToHost, ctx->st), "read");
                sync(ctx);
            } else {
                std::memcpy(dst, b + off, n);
            }
        };
        u64 h3[3];
        read_host(h3, 0, 24);
        fail_if(ctx, h3[0] != kVbMagic, LCG_EINVAL, "not a VByte grammar");
        const u64 k = h3[1], nl = h3[2];
        fail_if(ctx, k > 0xffffffffull || nl > 4096 || size < 24 + 32 * nl, LCG_EINVAL, "malformed VByte header");
        fail_if(ctx, nl >= ctx->levels, LCG_ELEVELS, "grammar has more levels than the hash family has functions");
        std::vector<u64> hd(4 * nl);
        read_host(hd.data(), 24, 32 * nl);
        std::vector<u64> off_len(nl), off_rhs(nl), off_F(nl);
        u64 pos = 24 + 32 * nl;
        for (u64 i = 0; i < nl; i++) {
            const u64 g = hd[4 * i], Gs = hd[4 * i + 1], nbl = hd[4 * i + 2], nbr = hd[4 * i + 3];
            fail_if(ctx, g > kMaxRank || Gs > (1ull << 40) || Gs < g || (g == 0) != (Gs == 0), LCG_EINVAL,
                    "malformed level sizes");
            fail_if(ctx, nbl < g || nbl > 5 * g || nbr < Gs || nbr > 5 * Gs, LCG_EINVAL,
                    "stream lengths do not fit the level sizes");
            off_len[i] = pos;
            pos += pad8(nbl);
            off_rhs[i] = pos;
            pos += pad8(nbr);
            off_F[i] = pos;
            pos += pad8(4 * g);
            fail_if(ctx, pos > size, LCG_EINVAL, "truncated");
        }
        const u64 off_cl = pos, off_cr = pos + pad8(4 * k), off_F0 = pos + 2 * pad8(4 * k);
        fail_if(ctx, off_F0 + 4 * 256 != size, LCG_EINVAL, "wrong size");
        // C entries name existing rules
        std::vector<uint32_t> cl(k), cr(k);
        read_host(cl.data(), off_cl, 4 * k);
        read_host(cr.data(), off_cr, 4 * k);
        for (u64 j = 0; j < k; j++) {
            fail_if(ctx, cl[j] > nl, LCG_EINVAL, "C entry " + std::to_string(j) + " names a missing level");
            const u64 lim = cl[j] == 0 ? 256 : hd[4 * (cl[j] - 1)];
            fail_if(ctx, cr[j] >= lim, LCG_EINVAL, "C entry " + std::to_string(j) + " names a missing rule");
        }
        const u8* src = b;
        if (!buf_on_device) {
            staging = dalloc<u8>(ctx, size);
            ck(ctx, cudaMemcpyAsync(staging, buf, size, cudaMemcpyHostToDevice, ctx->st), "upload");
            src = staging;
        }
        reset_status(ctx);
        G = new_grammar(ctx);
        if (k) {
            grow_c(ctx, G, (u32)k);
            ck(ctx, cudaMemcpyAsync(G->c_level, src + off_cl, 4 * k, cudaMemcpyDeviceToDevice, ctx->st), "import");
            ck(ctx, cudaMemcpyAsync(G->c_rank, src + off_cr, 4 * k, cudaMemcpyDeviceToDevice, ctx->st), "import");
            G->k = (u32)k;
        }
        // the levels' arrays, and one decode over all columns: every level's
        // rule lengths (into one array, scanned into the offsets afterwards)
        // and right-hand sides
        u64 sum_g = 0, max_g = 0;
        for (u64 i = 0; i < nl; i++) {
            sum_g += hd[4 * i];
            max_g = std::max<u64>(max_g, hd[4 * i]);
        }
        u32* lens = dalloc<u32>(ctx, sum_g);
        temps.push_back(lens);
        std::vector<VbDecCol> cols;
        std::vector<VbLevelOff> lvo;
        u64 T = 0, gbase = 0;
        for (u64 i = 0; i < nl; i++) {
            const u64 g = hd[4 * i], Gs = hd[4 * i + 1];
            G->lv.emplace_back();
            Level& L = G->lv.back();
            grow_level(ctx, L, g, Gs);
            L.g = g;
            L.G = Gs;
            L.rvalid = false;
            if (g == 0) continue;
            const u64 prev = i == 0 ? 256 : hd[4 * (i - 1)];
            cols.push_back(VbDecCol{src + off_len[i], hd[4 * i + 2], g, 1, 1ull << 32, lens + gbase, T});
            T += vb_decode_tiles(hd[4 * i + 2]);
            cols.push_back(VbDecCol{src + off_rhs[i], hd[4 * i + 3], Gs, 0, prev, L.rhs, T});
            T += vb_decode_tiles(hd[4 * i + 3]);
            lvo.push_back(VbLevelOff{L.rhs_off, g, Gs, gbase});
            gbase += g;
            ck(ctx, cudaMemcpyAsync(L.F, src + off_F[i], 4 * g, cudaMemcpyDeviceToDevice, ctx->st), "import");
        }
        const u32 ncols = (u32)cols.size();
        fail_if(ctx, ncols > (u32)kVbMaxCols, LCG_EINVAL, "too many levels");
        cols.push_back(VbDecCol{nullptr, 0, 0, 0, 0, nullptr, T});
        if (T) {
            VbDecCol* dcols = dalloc<VbDecCol>(ctx, cols.size());
            temps.push_back(dcols);
            VbLevelOff* dlvo = dalloc<VbLevelOff>(ctx, lvo.size());
            temps.push_back(dlvo);
            u32* cnt = dalloc<u32>(ctx, T);
            temps.push_back(cnt);
            u64* off = dalloc<u64>(ctx, T);
            temps.push_back(off);
            u64* gscan = dalloc<u64>(ctx, sum_g);
            temps.push_back(gscan);
            ck(ctx, cudaMemcpyAsync(dcols, cols.data(), sizeof(VbDecCol) * cols.size(), cudaMemcpyHostToDevice,
                                    ctx->st),
               "columns");
            ck(ctx, cudaMemcpyAsync(dlvo, lvo.data(), sizeof(VbLevelOff) * lvo.size(), cudaMemcpyHostToDevice,
                                    ctx->st),
               "levels");
            double nbytes = 0, nvals = 0;
            for (u32 c = 0; c < ncols; c++) {
                nbytes += (double)cols[c].nb;
                nvals += (double)cols[c].n;
            }
            int h = kt_begin(ctx, "k_vb_tile_ends", nbytes);
            ck(ctx, launch_vb_tile_ends_all(dcols, ncols, T, cnt, ctx->st), "k_vb_tile_ends");
            kt_end(ctx, h);
            vb_scan(ctx, cnt, T, off, ctx->scratch + 1);
            h = kt_begin(ctx, "k_vb_dwrite", nbytes + 4.0 * nvals);
            ck(ctx, launch_vb_dwrite_all(dcols, ncols, T, off, ctx->ds, ctx->st), "k_vb_dwrite");
            kt_end(ctx, h);
            vb_scan(ctx, lens, sum_g, gscan, ctx->scratch + 1);
            h = kt_begin(ctx, "k_vb_offsets", 12.0 * (double)sum_g);
            ck(ctx, launch_vb_offsets_all(dlvo, (u32)lvo.size(), max_g, gscan, ctx->scratch + 1, ctx->ds, ctx->st),
               "k_vb_offsets");
            kt_end(ctx, h);
            ctx->launches += 3;
        }
        // the streams are checked before anything reads what they gave
        DevStatus st = read_status(ctx);
        fail_if(ctx, st.error == kErrFormat, LCG_EINVAL, "malformed VByte form");
        check_device_status(ctx, st);
        for (u64 i = 0; i < nl; i++) {
            const Level& L = G->lv[i];
            ck(ctx, launch_check_fp(L.rhs, L.rhs_off, L.g, fprev_of(G, (u32)i + 1), level_hash(ctx, (u32)i + 1), L.F,
                                    ctx->ds, ctx->st),
               "k_check_fp");
            ctx->launches++;
        }
        uint32_t mine[256], theirs[256];
        ck(ctx, cudaMemcpyAsync(mine, G->F0, sizeof(mine), cudaMemcpyDeviceToHost, ctx->st), "read F0");
        ck(ctx, cudaMemcpyAsync(theirs, src + off_F0, sizeof(theirs), cudaMemcpyDeviceToHost, ctx->st), "read F0");
        dfree(ctx, staging);
        staging = nullptr;
        for (void* p : temps) dfree(ctx, p);
        temps.clear();
        st = read_status(ctx);
        kt_collect(ctx);
        fail_if(ctx, st.error == kErrMismatch, LCG_EMISMATCH,
                "imported fingerprints differ from those of this context's hash family");
        check_device_status(ctx, st);
        fail_if(ctx, std::memcmp(mine, theirs, sizeof(mine)) != 0, LCG_EMISMATCH,
                "VByte grammar: F0 of another hash family");
        *out = G;
        return LCG_OK;
    } catch (const Fail& f) {
        cudaStreamSynchronize(ctx->st);
        if (staging) cudaFree(staging);
        for (void* p : temps) cudaFree(p);
        free_grammar_now(G);
        return f.code;
    } catch (const std::bad_alloc&) {
        ctx->err = "host allocation failed";
        cudaStreamSynchronize(ctx->st);
        if (staging) cudaFree(staging);
        for (void* p : temps) cudaFree(p);
        free_grammar_now(G);
        return LCG_ENOMEM;
    }
}

void lcg_grammar_free(lcg_grammar* G) { free_grammar_now(G); }

int lcg_postprocess(lcg_ctx* ctx, const lcg_grammar* G, lcg_pp** out) {
    if (!ctx || !G || !out) return LCG_EINVAL;
    *out = nullptr;
    const Range range("lcg_postprocess");
    LCG_GUARD_BEGIN
    ck(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    fail_if(ctx, G->device != ctx->device, LCG_EINVAL, "grammar on another device");
    *out = postprocess(ctx, G);
    return LCG_OK;
    LCG_GUARD_END
}

int lcg_pp_stats_of(const lcg_pp* pp, lcg_pp_stats* out) {
    if (!pp || !out) return LCG_EINVAL;
    *out = pp->stats;
    return LCG_OK;
}

int lcg_pp_export(const lcg_pp* pp, uint8_t* kind, uint64_t* rhs_off, uint32_t* rhs, uint32_t* c) {
    if (!pp || !kind || !rhs_off || (!rhs && pp->size) || (!c && pp->k)) return LCG_EINVAL;
    if (cudaSetDevice(pp->device) != cudaSuccess) return LCG_EDEVICE;
    bool ok = cudaMemcpy(kind, pp->kind, pp->rules, cudaMemcpyDeviceToHost) == cudaSuccess &&
              cudaMemcpy(rhs_off, pp->rhs_off, 8 * (pp->rules + 1), cudaMemcpyDeviceToHost) == cudaSuccess;
    if (ok && pp->size) ok = cudaMemcpy(rhs, pp->rhs, 4 * pp->size, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (ok && pp->k) ok = cudaMemcpy(c, pp->c, 4ull * pp->k, cudaMemcpyDeviceToHost) == cudaSuccess;
    return ok ? LCG_OK : LCG_EDEVICE;
}

void lcg_pp_free(lcg_pp* pp) { free_pp(pp); }

}  // extern "C"
