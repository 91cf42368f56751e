/*
 * Plain CPU oracle of the stable locally consistent grammar (LCG) method.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct reference
 * that the GPU path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it; the product never does.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * What it computes (paper section / equation in brackets):
 *   - h^0 over bytes: ((a_0 s + b_0) mod p) mod m                     [Sec. 2.4, Sec. 3.2]
 *   - h^i over a phrase: ((a_i (sum_j F[Q_j] c_i^{j-1} mod p) + b_i) mod p) mod m
 *                                                                       [Eq. lvl_hash, Eq. fast_hash]
 *   - RandLMSPar types L/S/U and LMS breaks of each string              [Eq. rand_types, Sec. 3.3]
 *   - phrases = spans between consecutive breaks, string start a break  [Sec. 3.3, phrase definition]
 *   - BuildGram rounds: break, name distinct phrases, store rules,
 *     rewrite, retire strings of length one into C                     [Sec. 2.3 steps 1-4, Sec. 3.3]
 *   - MergeGrams level by level with the rank map M                    [Sec. 3.6]
 *   - expansion exp(C[j])                                               [Sec. 2.2]
 *
 * Readings of the paper this file takes:
 *   - p = 2^61-1 for every level; m = 2^m_bits (m_bits <= 32).  The parameters
 *     a_i, b_i, c_i are inputs (drawn by the seeded input generator).
 *   - Nonterminals of level i are 0-based ranks in first-occurrence order over
 *     the round's concatenated active strings (string index, then position).
 *   - The last position of a string, and any suffix run of fingerprint-equal
 *     symbols, has type U and never breaks; position 0 always starts a phrase.
 *   - Input strings of length one are compressed at once: C[j] = (level 0, byte).
 *     Empty strings are rejected.
 *   - Level-1 right-hand sides hold terminal byte values as uint32.
 *
 * Arithmetic is plain: products are formed in 128 bits and reduced with '%'.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define OG_P 2305843009213693951ull /* 2^61 - 1 */

enum { OG_OK = 0, OG_EINVAL = -1, OG_ENOMEM = -2, OG_ELEVELS = -3, OG_EMISMATCH = -4 };

/* ------------------------------------------------------------------------ */
/* growable arrays                                                           */
/* ------------------------------------------------------------------------ */

typedef struct { uint32_t* v; uint64_t n, cap; } vec32;
typedef struct { uint64_t* v; uint64_t n, cap; } vec64;

static int v32_push(vec32* a, uint32_t x) {
    if (a->n == a->cap) {
        uint64_t nc = a->cap ? a->cap * 2 : 16;
        uint32_t* p = (uint32_t*)realloc(a->v, nc * sizeof(uint32_t));
        if (!p) return OG_ENOMEM;
        a->v = p; a->cap = nc;
    }
    a->v[a->n++] = x;
    return OG_OK;
}
static int v64_push(vec64* a, uint64_t x) {
    if (a->n == a->cap) {
        uint64_t nc = a->cap ? a->cap * 2 : 16;
        uint64_t* p = (uint64_t*)realloc(a->v, nc * sizeof(uint64_t));
        if (!p) return OG_ENOMEM;
        a->v = p; a->cap = nc;
    }
    a->v[a->n++] = x;
    return OG_OK;
}

/* ------------------------------------------------------------------------ */
/* grammar                                                                   */
/* ------------------------------------------------------------------------ */

/* One level i >= 1: rule r has rhs[rhs_off[r] .. rhs_off[r+1]) over the ranks
 * of level i-1 (bytes at level 1) and fingerprint F[r] = h^i(rhs). */
typedef struct {
    vec64 rhs_off; /* g+1 entries, rhs_off[0] = 0 */
    vec32 rhs;
    vec32 F;
} og_level;

typedef struct {
    uint32_t F0[256];    /* h^0 of every byte */
    uint32_t nlevels;    /* number of levels >= 1 stored */
    og_level* lv;        /* lv[0] is level 1 */
    uint32_t k;
    uint32_t* c_level;   /* C[j] = (c_level[j], c_rank[j]) */
    uint32_t* c_rank;
    uint64_t hash_tag;   /* identifies the hash family (merge needs equal H) */
} og_grammar;

static uint64_t lv_g(const og_level* L) { return L->rhs_off.n ? L->rhs_off.n - 1 : 0; }

void og_free(og_grammar* G) {
    if (!G) return;
    for (uint32_t i = 0; i < G->nlevels; i++) {
        free(G->lv[i].rhs_off.v); free(G->lv[i].rhs.v); free(G->lv[i].F.v);
    }
    free(G->lv); free(G->c_level); free(G->c_rank); free(G);
}

static int og_add_level(og_grammar* G) {
    og_level* p = (og_level*)realloc(G->lv, (G->nlevels + 1) * sizeof(og_level));
    if (!p) return OG_ENOMEM;
    G->lv = p;
    memset(&G->lv[G->nlevels], 0, sizeof(og_level));
    G->nlevels++;
    return v64_push(&G->lv[G->nlevels - 1].rhs_off, 0);
}

static int og_add_rule(og_level* L, const uint32_t* q, uint64_t len, uint32_t fp) {
    for (uint64_t x = 0; x < len; x++)
        if (v32_push(&L->rhs, q[x])) return OG_ENOMEM;
    if (v64_push(&L->rhs_off, L->rhs.n)) return OG_ENOMEM;
    return v32_push(&L->F, fp);
}

/* ------------------------------------------------------------------------ */
/* hash family H (Sec. 3.2)                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    const uint64_t *a, *b, *c;
    uint32_t levels;
    uint64_t mmask; /* m - 1 */
} og_hash;

/* h^0(s) = ((a_0 s + b_0) mod p) mod m */
static uint32_t og_h0(const og_hash* H, uint32_t s) {
    u128 x = (u128)H->a[0] * s + H->b[0];
    return (uint32_t)((uint64_t)(x % OG_P) & H->mmask);
}

/* Eq. fast_hash: F[X] = ((a_i (sum_{j=1..q} F[Q_j] c_i^{j-1}) + b_i) mod p) mod m,
 * with fq[j-1] = F[Q_j].  The sum is evaluated term by term with a running
 * power c^{j-1}. */
static uint32_t og_hi(const og_hash* H, uint32_t i, const uint32_t* fq, uint64_t q) {
    uint64_t sum = 0, cp = 1;
    for (uint64_t j = 0; j < q; j++) {
        sum = (uint64_t)(((u128)fq[j] * cp + sum) % OG_P);
        cp = (uint64_t)(((u128)cp * H->c[i]) % OG_P);
    }
    u128 x = (u128)H->a[i] * sum + H->b[i];
    return (uint32_t)((uint64_t)(x % OG_P) & H->mmask);
}

static uint64_t og_family_tag(const og_hash* H) {
    /* FNV-1a over the parameters: used only to refuse merging grammars built
     * with different hash families. */
    uint64_t h = 1469598103934665603ull;
    for (uint32_t i = 0; i < H->levels; i++) {
        uint64_t w[3] = { H->a[i], H->b[i], H->c[i] };
        for (int t = 0; t < 3; t++)
            for (int by = 0; by < 8; by++) { h ^= (w[t] >> (8 * by)) & 0xff; h *= 1099511628211ull; }
    }
    h ^= H->mmask; h *= 1099511628211ull;
    return h;
}

/* ------------------------------------------------------------------------ */
/* RandLMSPar (Eq. rand_types) on one string of fingerprints                */
/* ------------------------------------------------------------------------ */

enum { T_U = 0, T_S = 1, T_L = 2 };

/* brk[l] = 1 iff a phrase starts at l: l = 0, or l is LMS-type (type S with
 * position l-1 of type L).  Types are computed right to left: the last
 * position is U; f[l] < f[l+1] gives S, f[l] > f[l+1] gives L, and equal
 * fingerprints (the relation ~) copy the type of l+1. */
int og_breaks(const uint32_t* f, uint64_t n, uint8_t* brk) {
    if (n == 0) return OG_OK;
    uint8_t* t = (uint8_t*)malloc(n);
    if (!t) return OG_ENOMEM;
    t[n - 1] = T_U;
    for (uint64_t l = n - 1; l-- > 0;) {
        if (f[l] < f[l + 1]) t[l] = T_S;
        else if (f[l] > f[l + 1]) t[l] = T_L;
        else t[l] = t[l + 1];
    }
    brk[0] = 1;
    for (uint64_t l = 1; l < n; l++) brk[l] = (t[l] == T_S && t[l - 1] == T_L);
    free(t);
    return OG_OK;
}

/* ------------------------------------------------------------------------ */
/* dictionary of phrases of one level: content -> rank                       */
/* (textbook open addressing with linear probing; keys are compared in full)*/
/* ------------------------------------------------------------------------ */

typedef struct {
    uint32_t* slot;      /* rank + 1, 0 = empty */
    uint64_t cap, used;
    const og_level* L;   /* contents live in the level's rules */
} og_dict;

static uint64_t og_content_hash(const uint32_t* q, uint64_t len) {
    uint64_t h = 1469598103934665603ull ^ len;
    for (uint64_t x = 0; x < len; x++) {
        for (int by = 0; by < 4; by++) { h ^= (q[x] >> (8 * by)) & 0xff; h *= 1099511628211ull; }
    }
    return h;
}

static int og_dict_init(og_dict* D, const og_level* L, uint64_t hint) {
    uint64_t cap = 64;
    while (cap < 2 * hint + 2) cap <<= 1;
    D->slot = (uint32_t*)calloc(cap, sizeof(uint32_t));
    if (!D->slot) return OG_ENOMEM;
    D->cap = cap; D->used = 0; D->L = L;
    return OG_OK;
}

static int og_rule_equals(const og_level* L, uint32_t r, const uint32_t* q, uint64_t len) {
    uint64_t s = L->rhs_off.v[r], e = L->rhs_off.v[r + 1];
    if (e - s != len) return 0;
    return memcmp(L->rhs.v + s, q, len * sizeof(uint32_t)) == 0;
}

/* returns rank or -1 */
static int64_t og_dict_find(const og_dict* D, const uint32_t* q, uint64_t len) {
    uint64_t i = og_content_hash(q, len) & (D->cap - 1);
    while (D->slot[i]) {
        uint32_t r = D->slot[i] - 1;
        if (og_rule_equals(D->L, r, q, len)) return r;
        i = (i + 1) & (D->cap - 1);
    }
    return -1;
}

static int og_dict_insert(og_dict* D, uint32_t r);

static int og_dict_grow(og_dict* D) {
    uint32_t* old = D->slot;
    uint64_t oc = D->cap;
    D->cap *= 2;
    D->slot = (uint32_t*)calloc(D->cap, sizeof(uint32_t));
    if (!D->slot) return OG_ENOMEM;
    D->used = 0;
    for (uint64_t i = 0; i < oc; i++)
        if (old[i] && og_dict_insert(D, old[i] - 1)) return OG_ENOMEM;
    free(old);
    return OG_OK;
}

static int og_dict_insert(og_dict* D, uint32_t r) {
    if (2 * (D->used + 1) > D->cap && og_dict_grow(D)) return OG_ENOMEM;
    const og_level* L = D->L;
    uint64_t s = L->rhs_off.v[r], e = L->rhs_off.v[r + 1];
    uint64_t i = og_content_hash(L->rhs.v + s, e - s) & (D->cap - 1);
    while (D->slot[i]) i = (i + 1) & (D->cap - 1);
    D->slot[i] = r + 1;
    D->used++;
    return OG_OK;
}

/* ------------------------------------------------------------------------ */
/* BuildGram (Sec. 3.3)                                                       */
/* ------------------------------------------------------------------------ */

int og_build(const uint8_t* data, const uint64_t* off, uint32_t k,
             const uint64_t* a, const uint64_t* b, const uint64_t* c, uint32_t nlev, uint32_t m_bits,
             og_grammar** out) {
    *out = NULL;
    if (k == 0 || nlev == 0 || m_bits == 0 || m_bits > 32) return OG_EINVAL;
    for (uint32_t j = 0; j < k; j++)
        if (off[j + 1] <= off[j]) return OG_EINVAL; /* empty string or bad offsets */

    og_hash H = { a, b, c, nlev, (m_bits == 32) ? 0xffffffffull : ((1ull << m_bits) - 1) };
    og_grammar* G = (og_grammar*)calloc(1, sizeof(og_grammar));
    if (!G) return OG_ENOMEM;
    G->k = k;
    G->hash_tag = og_family_tag(&H);
    G->c_level = (uint32_t*)calloc(k, sizeof(uint32_t));
    G->c_rank = (uint32_t*)calloc(k, sizeof(uint32_t));
    if (!G->c_level || !G->c_rank) { og_free(G); return OG_ENOMEM; }
    for (uint32_t s = 0; s < 256; s++) G->F0[s] = og_h0(&H, s);

    /* T^1: active strings as uint32 symbols; strings of length one are
     * compressed already (level 0). */
    vec32 cur = {0}, nxt = {0};
    vec64 cur_off = {0}, nxt_off = {0};
    vec32 cur_id = {0}, nxt_id = {0};
    int rc = OG_OK;
    v64_push(&cur_off, 0);
    for (uint32_t j = 0; j < k; j++) {
        uint64_t nj = off[j + 1] - off[j];
        if (nj == 1) { G->c_level[j] = 0; G->c_rank[j] = data[off[j]]; continue; }
        for (uint64_t x = off[j]; x < off[j + 1]; x++) v32_push(&cur, data[x]);
        v64_push(&cur_off, cur.n);
        v32_push(&cur_id, j);
    }

    uint32_t i = 1;
    vec32 f = {0};
    uint8_t* brk = NULL;
    while (cur_id.n > 0) {
        if (i >= nlev) { rc = OG_ELEVELS; break; }
        if ((rc = og_add_level(G))) break;
        og_level* L = &G->lv[i - 1];
        const uint32_t* Fprev = (i == 1) ? G->F0 : G->lv[i - 2].F.v;
        og_dict D;
        if ((rc = og_dict_init(&D, L, 1024))) break;
        nxt.n = 0; nxt_off.n = 0; nxt_id.n = 0;
        v64_push(&nxt_off, 0);
        for (uint64_t s = 0; s < cur_id.n && !rc; s++) {
            uint64_t lo = cur_off.v[s], hi = cur_off.v[s + 1], n = hi - lo;
            const uint32_t* S = cur.v + lo;
            /* fingerprints of the symbols: f[l] = F^{i-1}[T^i[l]] */
            f.n = 0;
            for (uint64_t l = 0; l < n; l++) v32_push(&f, Fprev[S[l]]);
            uint8_t* nb = (uint8_t*)realloc(brk, n);
            if (!nb) { rc = OG_ENOMEM; break; }
            brk = nb;
            og_breaks(f.v, n, brk);
            uint64_t start_len = nxt.n;
            for (uint64_t l = 0; l < n;) {
                uint64_t e = l + 1;
                while (e < n && !brk[e]) e++;
                int64_t r = og_dict_find(&D, S + l, e - l);
                if (r < 0) {
                    r = (int64_t)lv_g(L);
                    if (r >= 0xffffffffll) { rc = OG_EINVAL; break; }
                    if ((rc = og_add_rule(L, S + l, e - l, og_hi(&H, i, f.v + l, e - l)))) break;
                    if ((rc = og_dict_insert(&D, (uint32_t)r))) break;
                }
                v32_push(&nxt, (uint32_t)r);
                l = e;
            }
            if (rc) break;
            if (nxt.n - start_len == 1) {
                /* T^{i+1}_j has length one: the string is fully compressed */
                G->c_level[cur_id.v[s]] = i;
                G->c_rank[cur_id.v[s]] = nxt.v[start_len];
                nxt.n = start_len;
            } else {
                v64_push(&nxt_off, nxt.n);
                v32_push(&nxt_id, cur_id.v[s]);
            }
        }
        free(D.slot);
        if (rc) break;
        vec32 t32 = cur; cur = nxt; nxt = t32;
        vec64 t64 = cur_off; cur_off = nxt_off; nxt_off = t64;
        t32 = cur_id; cur_id = nxt_id; nxt_id = t32;
        i++;
    }
    free(cur.v); free(nxt.v); free(cur_off.v); free(nxt_off.v); free(cur_id.v); free(nxt_id.v);
    free(f.v); free(brk);
    if (rc) { og_free(G); return rc; }
    *out = G;
    return OG_OK;
}

/* ------------------------------------------------------------------------ */
/* MergeGrams (Sec. 3.6) with per-level 0-based ranks                        */
/* ------------------------------------------------------------------------ */

/* A absorbs B.  Level by level: B's rules (already over A's ranks of the
 * level below, via M) are looked up in a dictionary of A's rules; a hit maps
 * B's rank to A's, a miss appends the rule to A as the next rank.  The map M
 * of the level then rewrites B's rules of the level above and B's entries of
 * C at this level.  Finally C_A is extended by C_B.  Ranks are per level, so
 * the paper's shifts by L_a[i] / L_b[i] between global ids and ranks are the
 * identity here. */
int og_merge(og_grammar* A, const og_grammar* B) {
    if (A->hash_tag != B->hash_tag) return OG_EMISMATCH;
    for (int s = 0; s < 256; s++) if (A->F0[s] != B->F0[s]) return OG_EMISMATCH;
    int rc = OG_OK;
    uint32_t* Mprev = NULL; /* level 0: identity on bytes */
    uint32_t* Mcur = NULL;
    vec32 q = {0};
    uint32_t* cb_rank = (uint32_t*)malloc((B->k ? B->k : 1) * sizeof(uint32_t));
    if (!cb_rank) return OG_ENOMEM;
    memcpy(cb_rank, B->c_rank, B->k * sizeof(uint32_t));

    for (uint32_t i = 1; i <= B->nlevels && !rc; i++) {
        if (i > A->nlevels && (rc = og_add_level(A))) break;
        og_level* LA = &A->lv[i - 1];
        const og_level* LB = &B->lv[i - 1];
        uint64_t gb = lv_g(LB);
        og_dict D;
        if ((rc = og_dict_init(&D, LA, lv_g(LA) + gb))) break;
        for (uint64_t r = 0; r < lv_g(LA) && !rc; r++) rc = og_dict_insert(&D, (uint32_t)r);
        Mcur = (uint32_t*)malloc((gb ? gb : 1) * sizeof(uint32_t));
        if (!Mcur) { rc = OG_ENOMEM; free(D.slot); break; }
        for (uint64_t r = 0; r < gb && !rc; r++) {
            uint64_t s = LB->rhs_off.v[r], e = LB->rhs_off.v[r + 1];
            q.n = 0;
            for (uint64_t x = s; x < e; x++) v32_push(&q, Mprev ? Mprev[LB->rhs.v[x]] : LB->rhs.v[x]);
            int64_t ra = og_dict_find(&D, q.v, e - s);
            if (ra >= 0) {
                if (LA->F.v[ra] != LB->F.v[r]) { rc = OG_EMISMATCH; break; }
                Mcur[r] = (uint32_t)ra;
            } else {
                uint64_t nr = lv_g(LA);
                if ((rc = og_add_rule(LA, q.v, e - s, LB->F.v[r]))) break;
                Mcur[r] = (uint32_t)nr;
            }
        }
        free(D.slot);
        for (uint32_t j = 0; j < B->k; j++)
            if (B->c_level[j] == i) cb_rank[j] = Mcur[cb_rank[j]];
        free(Mprev);
        Mprev = Mcur; Mcur = NULL;
    }
    free(Mprev); free(Mcur); free(q.v);
    if (!rc) {
        uint32_t nk = A->k + B->k;
        uint32_t* cl = (uint32_t*)realloc(A->c_level, nk * sizeof(uint32_t));
        if (cl) A->c_level = cl;
        uint32_t* cr = (uint32_t*)realloc(A->c_rank, nk * sizeof(uint32_t));
        if (cr) A->c_rank = cr;
        if (!cl || !cr) rc = OG_ENOMEM;
        else {
            memcpy(A->c_level + A->k, B->c_level, B->k * sizeof(uint32_t));
            memcpy(A->c_rank + A->k, cb_rank, B->k * sizeof(uint32_t));
            A->k = nk;
        }
    }
    free(cb_rank);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* exp(C[j]) (Sec. 2.2)                                                       */
/* ------------------------------------------------------------------------ */

int og_decompress(const og_grammar* G, uint32_t j, uint8_t* out, uint64_t cap, uint64_t* out_len) {
    if (j >= G->k) return OG_EINVAL;
    /* explicit stack of (level, rank) */
    uint64_t scap = 64, sp = 0, n = 0;
    uint32_t* st = (uint32_t*)malloc(2 * scap * sizeof(uint32_t));
    if (!st) return OG_ENOMEM;
    st[0] = G->c_level[j]; st[1] = G->c_rank[j]; sp = 1;
    while (sp) {
        sp--;
        uint32_t lev = st[2 * sp], r = st[2 * sp + 1];
        if (lev == 0) {
            if (n < cap) out[n] = (uint8_t)r;
            n++;
            continue;
        }
        const og_level* L = &G->lv[lev - 1];
        uint64_t s = L->rhs_off.v[r], e = L->rhs_off.v[r + 1];
        if (sp + (e - s) > scap) {
            while (sp + (e - s) > scap) scap *= 2;
            uint32_t* ns = (uint32_t*)realloc(st, 2 * scap * sizeof(uint32_t));
            if (!ns) { free(st); return OG_ENOMEM; }
            st = ns;
        }
        for (uint64_t x = e; x-- > s;) { st[2 * sp] = lev - 1; st[2 * sp + 1] = L->rhs.v[x]; sp++; }
    }
    free(st);
    *out_len = n;
    return n <= cap ? OG_OK : OG_EINVAL;
}

/* ------------------------------------------------------------------------ */
/* accessors and construction from arrays (for the Python wrapper)           */
/* ------------------------------------------------------------------------ */

uint32_t og_nlevels(const og_grammar* G) { return G->nlevels; }
uint32_t og_k(const og_grammar* G) { return G->k; }
uint64_t og_level_g(const og_grammar* G, uint32_t i) { return lv_g(&G->lv[i - 1]); }
uint64_t og_level_G(const og_grammar* G, uint32_t i) { return G->lv[i - 1].rhs.n; }
const uint64_t* og_level_rhs_off(const og_grammar* G, uint32_t i) { return G->lv[i - 1].rhs_off.v; }
const uint32_t* og_level_rhs(const og_grammar* G, uint32_t i) { return G->lv[i - 1].rhs.v; }
const uint32_t* og_level_F(const og_grammar* G, uint32_t i) { return G->lv[i - 1].F.v; }
const uint32_t* og_F0(const og_grammar* G) { return G->F0; }
const uint32_t* og_c_level(const og_grammar* G) { return G->c_level; }
const uint32_t* og_c_rank(const og_grammar* G) { return G->c_rank; }
uint64_t og_hash_tag(const og_grammar* G) { return G->hash_tag; }

/* A grammar given level by level (used for hand-built merge fixtures and for
 * copies).  F0 and the family tag are taken as given. */
og_grammar* og_new(const uint32_t* F0, uint64_t tag, uint32_t k, const uint32_t* c_level, const uint32_t* c_rank) {
    og_grammar* G = (og_grammar*)calloc(1, sizeof(og_grammar));
    if (!G) return NULL;
    memcpy(G->F0, F0, sizeof(G->F0));
    G->hash_tag = tag;
    G->k = k;
    G->c_level = (uint32_t*)calloc(k ? k : 1, sizeof(uint32_t));
    G->c_rank = (uint32_t*)calloc(k ? k : 1, sizeof(uint32_t));
    if (!G->c_level || !G->c_rank) { og_free(G); return NULL; }
    memcpy(G->c_level, c_level, k * sizeof(uint32_t));
    memcpy(G->c_rank, c_rank, k * sizeof(uint32_t));
    return G;
}

int og_push_level(og_grammar* G, uint64_t g, const uint64_t* rhs_off, const uint32_t* rhs, const uint32_t* F) {
    int rc = og_add_level(G);
    if (rc) return rc;
    og_level* L = &G->lv[G->nlevels - 1];
    for (uint64_t r = 0; r < g; r++)
        if ((rc = og_add_rule(L, rhs + rhs_off[r], rhs_off[r + 1] - rhs_off[r], F[r]))) return rc;
    return OG_OK;
}

/* The family tag of a hash family, so that hand-built grammars can carry it. */
uint64_t og_family_tag_of(const uint64_t* a, const uint64_t* b, const uint64_t* c, uint32_t nlev, uint32_t m_bits) {
    og_hash H = { a, b, c, nlev, (m_bits == 32) ? 0xffffffffull : ((1ull << m_bits) - 1) };
    return og_family_tag(&H);
}
