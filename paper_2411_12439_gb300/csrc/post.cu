// Post-processing of a finished level grammar: run-length rules (RL) and
// grammar simplification (Simp) (Sec. 2.2, post-processing paragraph; run on
// the output of BuildGram, first RL, then Simp, Sec. 4).
//
// RL, per level: every maximal run Y^l (l >= 2) inside one right-hand side
// becomes a reference to the run-length rule (Y, l) of the level; the distinct
// pairs of a level are numbered in order of first occurrence (rule rank, then
// position).  Simp: a rule that occurs exactly once in the right-hand sides of
// the level above, and is neither a string's root nor the base of a run-length
// rule, is removed and its occurrence replaced by its right-hand side.
//
// The output is one grammar over global ids: bytes 0..255, then level by
// level the surviving rules (rank order) followed by the level's run-length
// rules.  A run-length rule is stored as [base id, run length] with kind 1.
//
// Kernels here take one thread per rule: right-hand sides are short, and a
// rule's runs never cross its boundaries.  The host side (abi.cu) runs them
// level by level with the library's scans in between.
#include "lcg_dev.cuh"
#include "lcg_internal.h"

namespace lcg {

constexpr u32 kRLFlag = 1u << 31;  // an RL-rewritten entry naming a run-length rule
constexpr u64 kPPEmpty = ~0ull;

static unsigned pp_grid(u64 n) {
    u64 b = (n + 255) / 256;
    if (b == 0) b = 1;
    const u64 cap = 152ull * 64;
    return (unsigned)(b < cap ? b : cap);
}

// Runs of rule r: out_len[r] = runs, rl_len[r] = runs of length >= 2.
__global__ void k_rl_count(const u64* __restrict__ off, const u32* __restrict__ rhs, u64 g, u32* out_len,
                           u32* rl_len) {
    for (u64 r = blockIdx.x * (u64)blockDim.x + threadIdx.x; r < g; r += (u64)gridDim.x * blockDim.x) {
        const u64 a = off[r], b = off[r + 1];
        u32 runs = 0, long_runs = 0;
        u64 p = a;
        while (p < b) {
            const u32 y = rhs[p];
            u64 e = p + 1;
            while (e < b && rhs[e] == y) e++;
            runs++;
            long_runs += (e - p >= 2) ? 1u : 0u;
            p = e;
        }
        out_len[r] = runs;
        rl_len[r] = long_runs;
    }
}

__device__ __forceinline__ u64 pp_key(u32 y, u64 len) { return ((u64)y << 32) | len; }

__device__ __forceinline__ u64 pp_home(u64 key, u64 mask) { return fmix64(key) & mask; }

// The slot of `key` in the run table (claimed when absent); ~0 when the
// table is full.
__device__ u64 pp_claim(u64* keys, u64 mask, u64 key) {
    u64 s = pp_home(key, mask);
    for (u64 probe = 0; probe <= mask; probe++) {
        const u64 old = atomicCAS((unsigned long long*)&keys[s], (unsigned long long)kPPEmpty,
                                  (unsigned long long)key);
        if (old == kPPEmpty || old == key) return s;
        s = (s + 1) & mask;
    }
    return ~0ull;
}

// Rewrite rule r: one entry per run (the symbol, or a placeholder for a run
// of length >= 2, listed with its symbol, length and output position; its
// (symbol, length) pair keeps the smallest list index in the run table).
__global__ void k_rl_write(const u64* __restrict__ off, const u32* __restrict__ rhs, u64 g,
                           const u64* __restrict__ new_off, const u64* __restrict__ rl_off, u32* new_rhs,
                           u32* run_y, u32* run_len, u64* run_pos, u64* keys, u64* vals, u64 mask, DevStatus* ds) {
    for (u64 r = blockIdx.x * (u64)blockDim.x + threadIdx.x; r < g; r += (u64)gridDim.x * blockDim.x) {
        const u64 a = off[r], b = off[r + 1];
        u64 w = new_off[r], m = rl_off[r];
        u64 p = a;
        while (p < b) {
            const u32 y = rhs[p];
            u64 e = p + 1;
            while (e < b && rhs[e] == y) e++;
            if (e - p >= 2) {
                run_y[m] = y;
                run_len[m] = (u32)(e - p);
                run_pos[m] = w;
                const u64 s = pp_claim(keys, mask, pp_key(y, e - p));
                if (s == ~0ull) set_error(ds, kErrTableFull);
                else atomicMin((unsigned long long*)&vals[s], (unsigned long long)m);
                new_rhs[w] = kRLFlag;  // named by k_rl_fix
                m++;
            } else {
                new_rhs[w] = y;
            }
            w++;
            p = e;
        }
    }
}

// first[m] = 1 when run m is the first of its (symbol, length) pair;
// run_first[m] = the list index of that first run.
__global__ void k_rl_first(const u32* __restrict__ run_y, const u32* __restrict__ run_len, u64 R,
                           const u64* __restrict__ keys, const u64* __restrict__ vals, u64 mask, u32* first,
                           u64* run_first, DevStatus* ds) {
    for (u64 m = blockIdx.x * (u64)blockDim.x + threadIdx.x; m < R; m += (u64)gridDim.x * blockDim.x) {
        const u64 key = pp_key(run_y[m], run_len[m]);
        u64 s = pp_home(key, mask);
        u64 f = ~0ull;
        for (u64 probe = 0; probe <= mask; probe++) {
            const u64 k = keys[s];
            if (k == key) { f = vals[s]; break; }
            if (k == kPPEmpty) break;
            s = (s + 1) & mask;
        }
        if (f == ~0ull) {
            set_error(ds, kErrTableFull);
            f = m;
        }
        run_first[m] = f;
        first[m] = (f == m) ? 1u : 0u;
    }
}

// Name every run: RL rule ids follow the first occurrences in list order.
__global__ void k_rl_fix(const u32* __restrict__ run_y, const u32* __restrict__ run_len,
                         const u64* __restrict__ run_pos, const u64* __restrict__ run_first,
                         const u64* __restrict__ rank_of, u64 R, u32* new_rhs, u32* rl_y, u32* rl_l, DevStatus* ds) {
    for (u64 m = blockIdx.x * (u64)blockDim.x + threadIdx.x; m < R; m += (u64)gridDim.x * blockDim.x) {
        const u64 f = run_first[m];
        const u64 id = rank_of[f];
        if (id >= (u64)kRLFlag) {
            set_error(ds, kErrRankOverflow);
            continue;
        }
        new_rhs[run_pos[m]] = kRLFlag | (u32)id;
        if (f == m) {
            rl_y[id] = run_y[m];
            rl_l[id] = run_len[m];
        }
    }
}

// Uses of the rules of the level below in the RL-rewritten right-hand sides
// of this level; bases of this level's run-length rules are kept.
__global__ void k_pp_uses(const u64* __restrict__ off, const u32* __restrict__ rhs, u64 g, u32* uses_below) {
    for (u64 r = blockIdx.x * (u64)blockDim.x + threadIdx.x; r < g; r += (u64)gridDim.x * blockDim.x) {
        for (u64 p = off[r]; p < off[r + 1]; p++) {
            const u32 v = rhs[p];
            if (!(v & kRLFlag)) atomicAdd(&uses_below[v], 1u);
        }
    }
}

__global__ void k_pp_pin_bases(const u32* __restrict__ rl_y, u64 nrl, u8* pinned_below) {
    for (u64 x = blockIdx.x * (u64)blockDim.x + threadIdx.x; x < nrl; x += (u64)gridDim.x * blockDim.x)
        pinned_below[rl_y[x]] = 1;
}

__global__ void k_pp_pin_roots(const u32* __restrict__ c_level, const u32* __restrict__ c_rank, u32 k,
                               PPLevels lv) {
    for (u64 j = blockIdx.x * (u64)blockDim.x + threadIdx.x; j < k; j += (u64)gridDim.x * blockDim.x) {
        const u32 l = c_level[j];
        if (l >= 1 && l <= lv.n) lv.pinned[l - 1][c_rank[j]] = 1;
    }
}

// surv[r] = 1 unless rule r is used exactly once and not kept.
__global__ void k_pp_survive(const u32* __restrict__ uses, const u8* __restrict__ pinned, u64 g, u32* surv) {
    for (u64 r = blockIdx.x * (u64)blockDim.x + threadIdx.x; r < g; r += (u64)gridDim.x * blockDim.x)
        surv[r] = (uses[r] == 1 && !pinned[r]) ? 0u : 1u;
}

// Length of rule r of level `li` (0-based) once removed rules below are
// expanded; the lengths of the level below are already known.  Surviving
// rules write it at their place in the output order.
__global__ void k_pp_explen(PPLevels lv, u32 li, u32* fin_len, DevStatus* ds) {
    const u64* off = lv.off[li];
    const u32* rhs = lv.rhs[li];
    const u64 g = lv.g[li];
    for (u64 r = blockIdx.x * (u64)blockDim.x + threadIdx.x; r < g; r += (u64)gridDim.x * blockDim.x) {
        u64 len = 0;
        for (u64 p = off[r]; p < off[r + 1]; p++) {
            const u32 v = rhs[p];
            if (li > 0 && !(v & kRLFlag) && !lv.surv[li - 1][v]) len += lv.explen[li - 1][v];
            else len += 1;
        }
        if (len > 0xffffffffull) {
            set_error(ds, kErrRankOverflow);
            len = 0;
        }
        lv.explen[li][r] = (u32)len;
        if (lv.surv[li][r]) fin_len[lv.base[li] - 256 + lv.spre[li][r]] = (u32)len;
    }
}

__global__ void k_pp_rl_len(PPLevels lv, u32 li, u32* fin_len) {
    const u64 nrl = lv.nrl[li];
    for (u64 x = blockIdx.x * (u64)blockDim.x + threadIdx.x; x < nrl; x += (u64)gridDim.x * blockDim.x)
        fin_len[lv.base[li] - 256 + lv.S[li] + x] = 2u;
}

// Final id of a plain symbol v of level li (0 = bytes).
__device__ __forceinline__ u32 pp_id(const PPLevels& lv, u32 li, u32 v) {
    return li == 0 ? v : (u32)(lv.base[li - 1] + lv.spre[li - 1][v]);
}

// Right-hand sides, top level first: a surviving rule writes its entries at
// its place in the output, a removed rule at the place its single use gave it
// (set by the pass over the level above).  An entry naming a removed rule of
// the level below reserves that rule's expanded length and hands it the
// position.  Every thread writes only its own rule's entries.
__global__ void k_pp_place(PPLevels lv, u32 li, const u64* __restrict__ fin_off, u32* out, u8* kind, DevStatus* ds) {
    const u64 g = lv.g[li];
    const u64* off = lv.off[li];
    const u32* rhs = lv.rhs[li];
    for (u64 r = blockIdx.x * (u64)blockDim.x + threadIdx.x; r < g; r += (u64)gridDim.x * blockDim.x) {
        u64 w, w_end;
        if (lv.surv[li][r]) {
            const u64 id = lv.base[li] - 256 + lv.spre[li][r];
            kind[id] = 0;
            w = fin_off[id];
            w_end = fin_off[id + 1];
        } else {
            w = lv.dst[li][r];
            w_end = w + lv.explen[li][r];
        }
        if (w == ~0ull) continue;  // only after an error above
        for (u64 p = off[r]; p < off[r + 1]; p++) {
            const u32 v = rhs[p];
            u64 len = 1;
            if (!(v & kRLFlag) && li > 0 && !lv.surv[li - 1][v]) {
                lv.dst[li - 1][v] = w;
                len = lv.explen[li - 1][v];
            } else if (w < w_end) {
                out[w] = (v & kRLFlag) ? (u32)(lv.base[li] + lv.S[li] + (v & ~kRLFlag)) : pp_id(lv, li, v);
            }
            w += len;
        }
        if (w != w_end) set_error(ds, kErrCapacity);
    }
}

__global__ void k_pp_write_rl(PPLevels lv, u32 li, const u64* __restrict__ fin_off, u32* out, u8* kind) {
    const u64 nrl = lv.nrl[li];
    for (u64 x = blockIdx.x * (u64)blockDim.x + threadIdx.x; x < nrl; x += (u64)gridDim.x * blockDim.x) {
        const u64 id = lv.base[li] - 256 + lv.S[li] + x;
        kind[id] = 1;
        const u64 w = fin_off[id];
        out[w] = pp_id(lv, li, lv.rl_y[li][x]);
        out[w + 1] = lv.rl_l[li][x];
    }
}

__global__ void k_pp_roots(const u32* __restrict__ c_level, const u32* __restrict__ c_rank, u32 k, PPLevels lv,
                           u32* c_out) {
    for (u64 j = blockIdx.x * (u64)blockDim.x + threadIdx.x; j < k; j += (u64)gridDim.x * blockDim.x)
        c_out[j] = pp_id(lv, c_level[j], c_rank[j]);
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------

cudaError_t launch_rl_count(const u64* off, const u32* rhs, u64 g, u32* out_len, u32* rl_len, cudaStream_t st) {
    k_rl_count<<<pp_grid(g), 256, 0, st>>>(off, rhs, g, out_len, rl_len);
    return cudaGetLastError();
}

cudaError_t launch_rl_write(const u64* off, const u32* rhs, u64 g, const u64* new_off, const u64* rl_off, u32* new_rhs,
                            u32* run_y, u32* run_len, u64* run_pos, u64* keys, u64* vals, u64 mask, DevStatus* ds,
                            cudaStream_t st) {
    k_rl_write<<<pp_grid(g), 256, 0, st>>>(off, rhs, g, new_off, rl_off, new_rhs, run_y, run_len, run_pos, keys, vals,
                                           mask, ds);
    return cudaGetLastError();
}

cudaError_t launch_rl_first(const u32* run_y, const u32* run_len, u64 R, const u64* keys, const u64* vals, u64 mask,
                            u32* first, u64* run_first, DevStatus* ds, cudaStream_t st) {
    if (R == 0) return cudaSuccess;
    k_rl_first<<<pp_grid(R), 256, 0, st>>>(run_y, run_len, R, keys, vals, mask, first, run_first, ds);
    return cudaGetLastError();
}

cudaError_t launch_rl_fix(const u32* run_y, const u32* run_len, const u64* run_pos, const u64* run_first,
                          const u64* rank_of, u64 R, u32* new_rhs, u32* rl_y, u32* rl_l, DevStatus* ds,
                          cudaStream_t st) {
    if (R == 0) return cudaSuccess;
    k_rl_fix<<<pp_grid(R), 256, 0, st>>>(run_y, run_len, run_pos, run_first, rank_of, R, new_rhs, rl_y, rl_l, ds);
    return cudaGetLastError();
}

cudaError_t launch_pp_uses(const u64* off, const u32* rhs, u64 g, u32* uses_below, cudaStream_t st) {
    k_pp_uses<<<pp_grid(g), 256, 0, st>>>(off, rhs, g, uses_below);
    return cudaGetLastError();
}

cudaError_t launch_pp_pin_bases(const u32* rl_y, u64 nrl, u8* pinned_below, cudaStream_t st) {
    if (nrl == 0) return cudaSuccess;
    k_pp_pin_bases<<<pp_grid(nrl), 256, 0, st>>>(rl_y, nrl, pinned_below);
    return cudaGetLastError();
}

cudaError_t launch_pp_pin_roots(const u32* c_level, const u32* c_rank, u32 k, const PPLevels& lv, cudaStream_t st) {
    if (k == 0) return cudaSuccess;
    k_pp_pin_roots<<<pp_grid(k), 256, 0, st>>>(c_level, c_rank, k, lv);
    return cudaGetLastError();
}

cudaError_t launch_pp_survive(const u32* uses, const u8* pinned, u64 g, u32* surv, cudaStream_t st) {
    k_pp_survive<<<pp_grid(g), 256, 0, st>>>(uses, pinned, g, surv);
    return cudaGetLastError();
}

cudaError_t launch_pp_lengths(const PPLevels& lv, u32 li, u32* fin_len, DevStatus* ds, cudaStream_t st) {
    k_pp_explen<<<pp_grid(lv.g[li]), 256, 0, st>>>(lv, li, fin_len, ds);
    if (lv.nrl[li]) k_pp_rl_len<<<pp_grid(lv.nrl[li]), 256, 0, st>>>(lv, li, fin_len);
    return cudaGetLastError();
}

cudaError_t launch_pp_write(const PPLevels& lv, u32 li, const u64* fin_off, u32* out, u8* kind, DevStatus* ds,
                            cudaStream_t st) {
    k_pp_place<<<pp_grid(lv.g[li]), 256, 0, st>>>(lv, li, fin_off, out, kind, ds);
    if (lv.nrl[li]) k_pp_write_rl<<<pp_grid(lv.nrl[li]), 256, 0, st>>>(lv, li, fin_off, out, kind);
    return cudaGetLastError();
}

cudaError_t launch_pp_roots(const u32* c_level, const u32* c_rank, u32 k, const PPLevels& lv, u32* c_out,
                            cudaStream_t st) {
    if (k == 0) return cudaSuccess;
    k_pp_roots<<<pp_grid(k), 256, 0, st>>>(c_level, c_rank, k, lv, c_out);
    return cudaGetLastError();
}

}  // namespace lcg
