// Host-side declarations shared by the translation units of the library
// (launchers of the kernels and the argument blocks they take).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "lcg_dev.cuh"

namespace lcg {

// Counts written by k_strings for the host.
struct RoundCounts {
    u64 phrases;  // phrases of the round (= |T^{i+1}| before retiring)
    u64 retired;  // strings that became one symbol
    u64 k_next;   // strings still active
    u64 n_next;   // |T^{i+1}|
};

struct RoundArgs {
    int sym_bytes;        // 1 in round 1 (bytes), 4 afterwards (ranks)
    const void* S;        // T^i
    u64 n;                // |T^i|
    const u64* soff;      // k+1 string offsets into T^i
    const u32* sid;       // original string index of each active string
    u32 k;
    const u32* Fprev;     // F^{i-1}
    LevelHash lh;         // parameters of h^i
    u32 level;            // i
    // break pass
    u32* bitmap;
    u64* tile_base;
    void* lb1;
    void* lb2;
    u64 epoch;
    u64* ctr;
    u64 ctr_base;
    u64* total;           // device: phrases of the round
    DevStatus* ds;
    // strings pass
    u64* soff_next;
    u32* sid_next;
    u64* R_phr;
    u32* R_sid;
    RoundCounts* rc;
    // phrase pass
    void* tab;
    u64 mask;
    u64 claim_limit;
    const void* rtab;     // resident table of level i (read), or null
    u64 rmask;
    const u32* rrhs;
    const u64* rrhs_off;
    u32* P_slot;
    // naming pass
    u64 P;                // phrases (host copy)
    u64 g_base, G_base;   // rules / rhs symbols of level i before this round
    u32* rhs;
    u64* rhs_off;
    u32* F;
    u64* totals;
    void* rtab_w;         // resident table of level i to extend, or null
    u64 rmask_w;
    // rewrite pass
    u32* Tnext;
    u32* c_level;
    u32* c_rank;
};

u64 tiles_for(u64 n);
u64 name_tiles_for(u64 P);
size_t lb1_bytes(u64 tiles);
size_t lb2_bytes(u64 tiles);
size_t slot_bytes();

cudaError_t launch_breaks(const RoundArgs& a, cudaStream_t st);
cudaError_t launch_strings(const RoundArgs& a, cudaStream_t st);
cudaError_t launch_phrases(const RoundArgs& a, cudaStream_t st);
cudaError_t launch_name(const RoundArgs& a, cudaStream_t st);
cudaError_t launch_rewrite(const RoundArgs& a, cudaStream_t st);
cudaError_t launch_level0(const unsigned char* data, const u64* pos, const u32* ids, u32 cnt, u32* c_level,
                          u32* c_rank, cudaStream_t st);
cudaError_t launch_resident_build(const u32* rhs, const u64* rhs_off, u64 r0, u64 cnt, const u32* Fprev,
                                  LevelHash lh, void* rtab, u64 rmask, DevStatus* ds, cudaStream_t st);
cudaError_t launch_h0(LevelHash h0, u32* F0, cudaStream_t st);
cudaError_t launch_gather_strings(const unsigned char* data, const u64* src_off, const u64* dst_off, u32 k,
                                  unsigned char* out, cudaStream_t st);

// grammar.cu
cudaError_t launch_remap(const u32* in, u64 n, const u32* M, u32* out, cudaStream_t st);
cudaError_t launch_merge_lookup(const u32* brhs, const u64* brhs_off, const u32* bF, u64 gb, const u32* aFprev,
                                LevelHash lh, const void* atab, u64 amask, const u32* arhs, const u64* arhs_off,
                                const u32* aF, u32* M, u32* miss, u32* mlen, DevStatus* ds, cudaStream_t st);
cudaError_t launch_merge_append(const u32* brhs, const u64* brhs_off, const u32* bF, u64 gb, const u32* miss,
                                const u64* xrank, const u64* xlen, u64 ga, u64 Ga, u32* arhs, u64* arhs_off,
                                u32* aF, u32* M, u64 ga_new, u64 Ga_new, cudaStream_t st);
cudaError_t launch_remap_c(const u32* c_level, u32* c_rank, u32 k, u32 level, const u32* M, cudaStream_t st);
cudaError_t launch_rule_lens(const u32* cur, u64 cnt, const u64* rhs_off, u32* lens, cudaStream_t st);
cudaError_t launch_expand(const u32* cur, u64 cnt, const u64* offs, const u64* rhs_off, const u32* rhs, u32* next,
                          cudaStream_t st);
cudaError_t launch_to_bytes(const u32* cur, u64 cnt, unsigned char* out, cudaStream_t st);
cudaError_t launch_scan2(const u32* in0, const u32* in1, u64 n, u64* out0, u64* out1, u64* totals, void* lb,
                         u64 epoch, u64* ctr, u64 ctr_base, DevStatus* ds, cudaStream_t st, u64* grid_out);
u64 scan2_tiles_for(u64 n);
size_t scan2_lb_bytes(u64 tiles);

}  // namespace lcg
