/*
 * oracle.c -- plain, slow, obviously correct CPU reference of the calculus of
 * Henrio, Kessler and Li (arXiv 1910.11110).  TEST INFRASTRUCTURE ONLY: it is
 * loaded by tests/, by __graft_entry__.smoke() and by bench.py's cpu_baseline
 * and reference legs, never by the product path, and it shares no code,
 * header, table or generator with the CUDA library.
 *
 * Everything here steps one operation at a time, in program order, over a
 * store sigma that maps each variable to its validity pair.  Effects are
 * applied by unifying the pair with the effect's signature, exactly as the
 * paper defines them; no transfer table is precomputed.
 *
 * Parity pins (tests/test_oracle_*.py): worked examples of Sections 3.1, 3.2,
 * 3.4 and 4.3; Property Safety and Property Progress; Theorems Subject
 * reduction / Progress on random well-declared programs; the VectorPU flag
 * code of Fig. vectorpucoherence; brute-force path enumeration for If/While.
 * The partial-write projection `pw` and the handling of dropped annotations
 * are readings, not paper statements, and are pinned only by the per-element
 * array model of the tests.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Validity values and status pairs (Section 3.1).                           */
/* ------------------------------------------------------------------------ */
enum { I = 0, V = 1 };
enum { ST_F = 4 };                       /* stuck: no rule applies (Property Progress) */
enum { K_R = 0, K_W, K_PUSH, K_PULL, K_NOOP, K_PW, K_GT, K_EN,
       T_IF = 8, T_ELSE = 9, T_WHILE = 10, T_END = 11 };

typedef struct { int local, remote; } pair_t;   /* local = CPU, remote = GPU */

static pair_t decode(int code) { pair_t p = { code & 1, (code >> 1) & 1 }; return p; }
static int encode(pair_t p) { return p.local | (p.remote << 1); }

/* A term of an effect signature: a constant V or I, or one of the variables
 * X, Y that are universally quantified in each signature (Section 3.1). */
typedef struct { int is_var; int v; } term_t;      /* v: V/I, or 0 = X, 1 = Y */
#define CV { 0, V }
#define CI { 0, I }
#define TX { 1, 0 }
#define TY { 1, 1 }
typedef struct { term_t pre[2]; term_t post[2]; } effect_t;

/* Section 3.1 effect signatures, in op-byte kind order.  The sixth entry is the
 * partial-write projection onto an overlapping array: a reading (the paper has
 * element writes w x[i], Section 3.5); its own side keeps its validity and the
 * other side becomes invalid. */
static const effect_t EFFECT[6] = {
    /* r    : (V,X) |-> (V,X) */ { { CV, TX }, { CV, TX } },
    /* w    : (X,Y) |-> (V,I) */ { { TX, TY }, { CV, CI } },
    /* Push : (V,X) |-> (V,V) */ { { CV, TX }, { CV, CV } },
    /* Pull : (X,V) |-> (V,V) */ { { TX, CV }, { CV, CV } },
    /* Noop : (X,Y) |-> (X,Y) */ { { TX, TY }, { TX, TY } },
    /* pw   : (X,Y) |-> (X,I) */ { { TX, TY }, { TX, CI } },
};

/* Unification of a signature's pre-pattern with a concrete pair: instantiate
 * X and Y so that both become identical; fail if no instantiation exists
 * (Section 3.1: an effect applies only through such a unification). */
static int unify(const term_t pat[2], pair_t s, int bind[2])
{
    int val[2] = { s.local, s.remote };
    bind[0] = bind[1] = -1;
    for (int k = 0; k < 2; k++) {
        if (!pat[k].is_var) {
            if (pat[k].v != val[k]) return 0;
        } else {
            int x = pat[k].v;
            if (bind[x] >= 0 && bind[x] != val[k]) return 0;
            bind[x] = val[k];
        }
    }
    return 1;
}

static pair_t instantiate(const term_t pat[2], const int bind[2])
{
    pair_t p;
    p.local = pat[0].is_var ? bind[pat[0].v] : pat[0].v;
    p.remote = pat[1].is_var ? bind[pat[1].v] : pat[1].v;
    return p;
}

/* Rules Effect and Remote Effect of Fig. Opsem.  Returns 0 when stuck. */
static int effect_step(int kind, int remote, pair_t s, pair_t* out)
{
    const effect_t* e = &EFFECT[kind];
    int bind[2];
    if (!remote) {
        /* sigma(x) = (X,Y), E : (X,Y) |-> (Z,T)  gives  (Z,T) */
        if (!unify(e->pre, s, bind)) return 0;
        *out = instantiate(e->post, bind);
    } else {
        /* sigma(x) = (X,Y), E : (Y,X) |-> (Z,T)  gives  (T,Z) */
        pair_t swapped = { s.remote, s.local };
        if (!unify(e->pre, swapped, bind)) return 0;
        pair_t z = instantiate(e->post, bind);
        out->local = z.remote;
        out->remote = z.local;
    }
    return 1;
}

int oracle_apply(int kind, int side, int status)
{
    if (status == ST_F) return ST_F;           /* a stuck variable stays stuck */
    pair_t out;
    if (!effect_step(kind, side, decode(status), &out)) return ST_F;
    return encode(out);
}

/* Conditions of Fig. Opsem: isValid x reads the local flag, remIsValid x the
 * remote one.  A stuck variable has no pair; its condition is taken as false. */
static int is_valid_on(int side, int status)
{
    if (status == ST_F) return 0;
    pair_t p = decode(status);
    return side == 0 ? p.local == V : p.remote == V;
}

/* The transfer that restores validity on `side` in Fig. sem-AM: the CPU-side
 * declaration emits Pull, the GPU-side declaration emits Push, both as plain
 * (non-remote) statements. */
static int transfer_for(int side, int status)
{
    return oracle_apply(side == 0 ? K_PULL : K_PUSH, 0, status);
}

/* ------------------------------------------------------------------------ */
/* Trace mode                                                                */
/* ------------------------------------------------------------------------ */
static int valid_trace_byte(uint8_t ks) { return (ks & 0xE0) == 0 && (ks & 15) <= K_EN; }

int oracle_check_trace(const uint8_t* kind_side, const int32_t* var, int64_t n_ops,
                       int32_t n_vars, const uint8_t* init_status,
                       uint8_t* step_status, uint8_t* final_status,
                       int32_t* var_first_fault, int64_t* first_fault)
{
    if (n_ops < 0 || n_vars < 0 || n_ops > INT32_MAX) return -1;
    for (int64_t i = 0; i < n_ops; i++) {
        if (!valid_trace_byte(kind_side[i])) return -1;
        if (var[i] < 0 || var[i] >= n_vars) return -2;
        int k = kind_side[i] & 15;
        if (k == K_GT) {
            /* a guarded transfer is followed by the check on its guard variable */
            if (i + 1 >= n_ops || (kind_side[i + 1] & 15) != K_EN ||
                (kind_side[i + 1] >> 4) != (kind_side[i] >> 4) || var[i + 1] == var[i])
                return -1;
        }
    }
    uint8_t* st = (uint8_t*)malloc((size_t)(n_vars ? n_vars : 1));
    if (!st) return -3;
    for (int32_t v = 0; v < n_vars; v++) {
        st[v] = init_status ? init_status[v] : (uint8_t)encode((pair_t){ V, I });  /* sigma_0 */
        if (st[v] > ST_F) { free(st); return -1; }
        var_first_fault[v] = -1;
    }
    int64_t ff = -1;
    for (int64_t i = 0; i < n_ops; i++) {
        int k = kind_side[i] & 15, side = kind_side[i] >> 4;
        int v = var[i];
        int before = st[v], after;
        if (k <= K_PW) {
            after = oracle_apply(k, side, before);
        } else if (k == K_GT) {
            /* if (valid_side(guard)) Noop else transfer on the real variable */
            int guard = st[var[i + 1]];
            after = is_valid_on(side, guard) ? before : transfer_for(side, before);
        } else { /* K_EN: the same test on the abstract variable itself */
            after = is_valid_on(side, before) ? before : transfer_for(side, before);
        }
        st[v] = (uint8_t)after;
        step_status[i] = (uint8_t)after;
        if (after == ST_F && before != ST_F) {
            if (var_first_fault[v] < 0) var_first_fault[v] = (int32_t)i;
            if (ff < 0) ff = i;
        }
    }
    for (int32_t v = 0; v < n_vars; v++) final_status[v] = st[v];
    *first_fault = ff;
    free(st);
    return 0;
}

/* The same check restricted to the variables v with v % n_shards == shard:
 * every op is read, ops on other variables are skipped (a variable's statuses
 * depend only on its own ops, Fig. Opsem rules Effect / Remote Effect), and
 * only the outputs of those variables are written: step_status at their
 * positions, final_status / var_first_fault at their ids, *first_fault = the
 * smallest of their first faults.  Used to run the oracle on several host
 * threads at once; traces with GT are rejected (-1). */
int oracle_check_trace_shard(const uint8_t* kind_side, const int32_t* var, int64_t n_ops,
                             int32_t n_vars, int32_t n_shards, int32_t shard,
                             uint8_t* step_status, uint8_t* final_status,
                             int32_t* var_first_fault, int64_t* first_fault)
{
    if (n_ops < 0 || n_vars < 0 || n_ops > INT32_MAX || n_shards < 1 || shard < 0 || shard >= n_shards)
        return -1;
    uint8_t* st = (uint8_t*)malloc((size_t)(n_vars ? n_vars : 1));
    if (!st) return -3;
    for (int32_t v = shard; v < n_vars; v += n_shards) {
        st[v] = (uint8_t)encode((pair_t){ V, I });                          /* sigma_0 */
        var_first_fault[v] = -1;
    }
    int64_t ff = -1;
    for (int64_t i = 0; i < n_ops; i++) {
        const int32_t v = var[i];
        if (v < 0 || v >= n_vars) { free(st); return -2; }
        if (v % n_shards != shard) continue;
        if (!valid_trace_byte(kind_side[i]) || (kind_side[i] & 15) > K_PW) { free(st); return -1; }
        int k = kind_side[i] & 15, side = kind_side[i] >> 4;
        int before = st[v], after = oracle_apply(k, side, before);
        st[v] = (uint8_t)after;
        step_status[i] = (uint8_t)after;
        if (after == ST_F && before != ST_F) {
            if (var_first_fault[v] < 0) var_first_fault[v] = (int32_t)i;
            if (ff < 0) ff = i;
        }
    }
    for (int32_t v = shard; v < n_vars; v += n_shards) final_status[v] = st[v];
    *first_fault = ff;
    free(st);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Relation mode: status sets, If = union of branches, While = closure       */
/* ------------------------------------------------------------------------ */
typedef struct {
    const uint8_t* tok;
    const int32_t* payload;
    int32_t n_vars;
    uint8_t* step_mask;
    int64_t first_fault;           /* relative token index, -1 none */
    int depth;
} prog_ctx;

#define ORACLE_MAX_DEPTH 64

static uint8_t image(int kind, int side, uint8_t mask)
{
    uint8_t out = 0;
    for (int s = 0; s <= ST_F; s++)
        if (mask & (1u << s)) out |= (uint8_t)(1u << oracle_apply(kind, side, s));
    return out;
}

static int eval_seq(prog_ctx* c, int64_t lo, int64_t hi, uint8_t* mask);

static uint8_t* copy_masks(const prog_ctx* c, const uint8_t* m)
{
    uint8_t* out = (uint8_t*)malloc((size_t)(c->n_vars ? c->n_vars : 1));
    if (out) memcpy(out, m, (size_t)c->n_vars);
    return out;
}

static int eval_seq(prog_ctx* c, int64_t lo, int64_t hi, uint8_t* mask)
{
    if (++c->depth > ORACLE_MAX_DEPTH) return -1;
    int64_t i = lo;
    while (i < hi) {
        int k = c->tok[i] & 15, side = (c->tok[i] >> 4) & 1;
        if ((c->tok[i] & 0xE0) != 0) return -1;
        if (k <= K_PW) {
            int32_t v = c->payload[i];
            if (v < 0 || v >= c->n_vars) return -2;
            uint8_t pre = mask[v], post = image(k, side, pre);
            /* may-fault origin: a possible non-stuck status that gets stuck here */
            for (int s = 0; s < ST_F; s++)
                if ((pre & (1u << s)) && oracle_apply(k, side, s) == ST_F) {
                    if (c->first_fault < 0 || i < c->first_fault) c->first_fault = i;
                    break;
                }
            mask[v] = post;
            c->step_mask[i] = post;
            i++;
        } else if (k == T_IF) {
            int64_t lt = c->payload[i];
            int64_t e = i + 1 + lt;                       /* ELSE token */
            if (lt < 0 || e >= hi || c->tok[e] != T_ELSE || side) return -1;
            int64_t le = c->payload[e];
            int64_t end = e + 1 + le;                     /* END token */
            if (le < 0 || end >= hi || c->tok[end] != T_END) return -1;
            /* IF-True / IF-False: both branches start from the same store */
            uint8_t* m_then = copy_masks(c, mask);
            uint8_t* m_else = copy_masks(c, mask);
            if (!m_then || !m_else) { free(m_then); free(m_else); return -3; }
            int rc = eval_seq(c, i + 1, e, m_then);
            if (!rc) rc = eval_seq(c, e + 1, end, m_else);
            if (!rc)
                for (int32_t v = 0; v < c->n_vars; v++) mask[v] = m_then[v] | m_else[v];
            free(m_then);
            free(m_else);
            if (rc) return rc;
            c->step_mask[i] = c->step_mask[e] = c->step_mask[end] = 0;
            i = end + 1;
        } else if (k == T_WHILE) {
            int64_t lb = c->payload[i];
            int64_t end = i + 1 + lb;
            if (lb < 0 || end >= hi || c->tok[end] != T_END || side) return -1;
            /* While-True / While-False: the set of stores at the loop head is the
             * least X with X = entry U body(X); the body's step sets are those of
             * the pass that starts from that fixpoint. */
            uint8_t* x = copy_masks(c, mask);
            if (!x) return -3;
            for (;;) {
                uint8_t* y = copy_masks(c, x);
                if (!y) { free(x); return -3; }
                int rc = eval_seq(c, i + 1, end, y);
                if (rc) { free(x); free(y); return rc; }
                int changed = 0;
                for (int32_t v = 0; v < c->n_vars; v++) {
                    uint8_t u = x[v] | y[v];
                    if (u != x[v]) { x[v] = u; changed = 1; }
                }
                free(y);
                if (!changed) break;
            }
            memcpy(mask, x, (size_t)c->n_vars);
            free(x);
            c->step_mask[i] = c->step_mask[end] = 0;
            i = end + 1;
        } else {
            return -1;      /* ELSE / END without a matching IF / WHILE, or GT / EN */
        }
    }
    c->depth--;
    return 0;
}

int oracle_check_program(const uint8_t* tok, const int32_t* payload, int64_t n_tok,
                         int32_t n_vars, const uint8_t* init_mask,
                         uint8_t* step_mask, uint8_t* final_mask, int64_t* first_fault)
{
    if (n_tok < 0 || n_vars < 0) return -1;
    prog_ctx c = { tok, payload, n_vars, step_mask, -1, 0 };
    for (int32_t v = 0; v < n_vars; v++) {
        final_mask[v] = init_mask ? init_mask[v] : (uint8_t)(1u << encode((pair_t){ V, I }));
        if (final_mask[v] >> 5) return -1;
    }
    int rc = eval_seq(&c, 0, n_tok, final_mask);
    if (rc) return rc;
    *first_fault = c.first_fault;
    return 0;
}

int oracle_check_batch(const uint8_t* tok, const int32_t* payload, const int64_t* prog_tok_off,
                       const int32_t* prog_nvars, const int64_t* prog_var_off, int64_t n_progs,
                       uint8_t* step_mask, uint8_t* final_mask, int64_t* prog_first_fault)
{
    if (n_progs < 0 || prog_tok_off[0] != 0 || prog_var_off[0] != 0) return -1;
    for (int64_t p = 0; p < n_progs; p++) {
        int64_t t0 = prog_tok_off[p], t1 = prog_tok_off[p + 1];
        if (t1 < t0 || prog_var_off[p + 1] - prog_var_off[p] != prog_nvars[p]) return -1;
        int rc = oracle_check_program(tok + t0, payload + t0, t1 - t0, prog_nvars[p], NULL,
                                      step_mask + t0, final_mask + prog_var_off[p],
                                      &prog_first_fault[p]);
        if (rc) return rc;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Path-sensitive relation mode: the conditions isValid g and remIsValid g   */
/* of Fig. Opsem (rules valid / invalid / rem-valid / rem-invalid) evaluated  */
/* on one guard variable g per program, other conditions (x (+) y) opaque.   */
/* The state at a program point is, for every variable x other than g, the   */
/* set of reachable pairs (status of g, status of x) -- a 5x5 bit matrix,    */
/* bit 5 i + j for g = i, x = j -- and the set of reachable statuses of g.   */
/* Control flow depends on g alone, so these pair sets are exactly the       */
/* projections of the reachable stores (each variable's F absorbing and not  */
/* stopping the others, as in the opaque relation mode).  A condition on g   */
/* keeps, on each branch, the pairs whose g status makes it true / false; a  */
/* stuck g satisfies neither rule, so its paths end there.  While: the pairs */
/* at the loop head are the least X with X = entry U body(X restricted to    */
/* the condition); the loop leaves with X restricted to its negation.  Token */
/* byte of IF / WHILE: bits 4-5 = condition (0 opaque, 1 isValid g,         */
/* 2 remIsValid g).                                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    const uint8_t* tok;
    const int32_t* payload;
    int32_t n_vars, g;
    uint8_t* step_mask;
    int64_t first_fault;
    int depth;
} ps_ctx;

typedef struct {
    uint8_t G;                     /* statuses of g */
    uint32_t* J;                   /* [n_vars] pair sets (unused at g) */
} ps_state;

/* g statuses for which the condition holds (then) and fails (else) */
static void ps_rows(int cond, uint8_t* t_rows, uint8_t* e_rows)
{
    if (cond == 0) { *t_rows = *e_rows = 31; return; }       /* opaque: both, every path */
    uint8_t t = 0, e = 0;
    for (int s = 0; s < ST_F; s++) {                         /* F: no rule applies */
        if (is_valid_on(cond == 1 ? 0 : 1, s)) t |= (uint8_t)(1u << s);
        else e |= (uint8_t)(1u << s);
    }
    *t_rows = t;
    *e_rows = e;
}

static uint32_t ps_keep_rows(uint32_t J, uint8_t rows)
{
    uint32_t out = 0;
    for (int i = 0; i <= ST_F; i++)
        if (rows & (1u << i)) out |= J & (31u << (5 * i));
    return out;
}

static uint8_t ps_proj(uint32_t J)
{
    uint8_t m = 0;
    for (int i = 0; i <= ST_F; i++) m |= (uint8_t)((J >> (5 * i)) & 31u);
    return m;
}

static int ps_alloc(const ps_ctx* c, ps_state* d, const ps_state* src)
{
    d->J = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(c->n_vars ? c->n_vars : 1));
    if (!d->J) return -3;
    d->G = src->G;
    memcpy(d->J, src->J, sizeof(uint32_t) * (size_t)c->n_vars);
    return 0;
}

static void ps_restrict(const ps_ctx* c, ps_state* st, uint8_t rows)
{
    st->G &= rows;
    for (int32_t x = 0; x < c->n_vars; x++)
        if (x != c->g) st->J[x] = ps_keep_rows(st->J[x], rows);
}

static int ps_eval(ps_ctx* c, int64_t lo, int64_t hi, ps_state* st)
{
    if (++c->depth > ORACLE_MAX_DEPTH) return -1;
    int64_t i = lo;
    while (i < hi) {
        int k = c->tok[i] & 15, hb = c->tok[i] >> 4;
        if (k <= K_PW) {
            if (hb > 1) return -1;
            int side = hb;
            int32_t v = c->payload[i];
            if (v < 0 || v >= c->n_vars) return -2;
            uint8_t pre, post;
            if (v == c->g) {
                /* an op on g moves every pair's first component */
                pre = st->G;
                post = image(k, side, pre);
                for (int32_t x = 0; x < c->n_vars; x++) {
                    if (x == c->g) continue;
                    uint32_t out = 0;
                    for (int gi = 0; gi <= ST_F; gi++) {
                        uint32_t row = (st->J[x] >> (5 * gi)) & 31u;
                        if (row) out |= row << (5 * oracle_apply(k, side, gi));
                    }
                    st->J[x] = out;
                }
                st->G = post;
            } else {
                pre = ps_proj(st->J[v]);
                uint32_t out = 0;
                for (int gi = 0; gi <= ST_F; gi++)
                    out |= (uint32_t)image(k, side, (uint8_t)((st->J[v] >> (5 * gi)) & 31u)) << (5 * gi);
                st->J[v] = out;
                post = ps_proj(out);
            }
            for (int s = 0; s < ST_F; s++)
                if ((pre & (1u << s)) && oracle_apply(k, side, s) == ST_F) {
                    if (c->first_fault < 0 || i < c->first_fault) c->first_fault = i;
                    break;
                }
            c->step_mask[i] = post;
            i++;
        } else if (k == T_IF) {
            if (hb > 2 || (hb && c->g < 0)) return -1;
            int64_t lt = c->payload[i], e = i + 1 + lt;
            if (lt < 0 || e >= hi || c->tok[e] != T_ELSE) return -1;
            int64_t le = c->payload[e], end = e + 1 + le;
            if (le < 0 || end >= hi || c->tok[end] != T_END) return -1;
            uint8_t tr, er;
            ps_rows(hb, &tr, &er);
            ps_state other;
            int rc = ps_alloc(c, &other, st);
            if (rc) return rc;
            ps_restrict(c, st, tr);                          /* IF-True paths */
            ps_restrict(c, &other, er);                      /* IF-False paths */
            rc = ps_eval(c, i + 1, e, st);
            if (!rc) rc = ps_eval(c, e + 1, end, &other);
            if (!rc) {
                st->G |= other.G;
                for (int32_t x = 0; x < c->n_vars; x++) st->J[x] |= other.J[x];
            }
            free(other.J);
            if (rc) return rc;
            c->step_mask[i] = c->step_mask[e] = c->step_mask[end] = 0;
            i = end + 1;
        } else if (k == T_WHILE) {
            if (hb > 2 || (hb && c->g < 0)) return -1;
            int64_t lb = c->payload[i], end = i + 1 + lb;
            if (lb < 0 || end >= hi || c->tok[end] != T_END) return -1;
            uint8_t tr, er;
            ps_rows(hb, &tr, &er);
            /* loop head: least X with X = entry U body(X on While-True paths) */
            for (;;) {
                ps_state y;
                int rc = ps_alloc(c, &y, st);
                if (rc) return rc;
                ps_restrict(c, &y, tr);
                rc = ps_eval(c, i + 1, end, &y);
                if (rc) { free(y.J); return rc; }
                int changed = (uint8_t)(st->G | y.G) != st->G;
                st->G |= y.G;
                for (int32_t x = 0; x < c->n_vars; x++) {
                    uint32_t u = st->J[x] | y.J[x];
                    if (u != st->J[x]) { st->J[x] = u; changed = 1; }
                }
                free(y.J);
                if (!changed) break;
            }
            ps_restrict(c, st, er);                          /* While-False: the loop is left */
            c->step_mask[i] = c->step_mask[end] = 0;
            i = end + 1;
        } else {
            return -1;
        }
    }
    c->depth--;
    return 0;
}

int oracle_check_program_guarded(const uint8_t* tok, const int32_t* payload, int64_t n_tok, int32_t n_vars,
                                 int32_t guard, const uint8_t* init_mask, uint8_t* step_mask,
                                 uint8_t* final_mask, int64_t* first_fault)
{
    if (n_tok < 0 || n_vars < 0 || guard < -1 || guard >= n_vars) return -1;
    ps_ctx c = { tok, payload, n_vars, guard, step_mask, -1, 0 };
    ps_state st;
    st.J = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n_vars ? n_vars : 1));
    if (!st.J) return -3;
    uint8_t vi = (uint8_t)(1u << encode((pair_t){ V, I }));
    st.G = guard >= 0 ? (init_mask ? init_mask[guard] : vi) : 1;       /* no guard: one row */
    int rc = 0;
    for (int32_t x = 0; x < n_vars && !rc; x++) {
        uint8_t m = init_mask ? init_mask[x] : vi;
        if (m >> 5) rc = -1;
        st.J[x] = 0;
        for (int gi = 0; gi <= ST_F; gi++)
            if (st.G & (1u << gi)) st.J[x] |= (uint32_t)m << (5 * gi);
    }
    if (!rc) rc = ps_eval(&c, 0, n_tok, &st);
    if (!rc) {
        for (int32_t x = 0; x < n_vars; x++) final_mask[x] = x == guard ? st.G : ps_proj(st.J[x]);
        *first_fault = c.first_fault;
    }
    free(st.J);
    return rc;
}

int oracle_check_batch_guarded(const uint8_t* tok, const int32_t* payload, const int64_t* prog_tok_off,
                               const int32_t* prog_nvars, const int64_t* prog_var_off, const int32_t* prog_guard,
                               int64_t n_progs, uint8_t* step_mask, uint8_t* final_mask, int64_t* prog_first_fault)
{
    if (n_progs < 0 || prog_tok_off[0] != 0 || prog_var_off[0] != 0) return -1;
    for (int64_t p = 0; p < n_progs; p++) {
        int64_t t0 = prog_tok_off[p], t1 = prog_tok_off[p + 1];
        if (t1 < t0 || prog_var_off[p + 1] - prog_var_off[p] != prog_nvars[p]) return -1;
        int rc = oracle_check_program_guarded(tok + t0, payload + t0, t1 - t0, prog_nvars[p], prog_guard[p], NULL,
                                              step_mask + t0, final_mask + prog_var_off[p], &prog_first_fault[p]);
        if (rc) return rc;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* VectorPU calls over possibly overlapping arrays                           */
/* ------------------------------------------------------------------------ */
static int overlap(int32_t s1, int32_t l1, int32_t s2, int32_t l2)
{
    /* half-open intervals [s, s+l) share an element */
    return (int64_t)s1 < (int64_t)s2 + l2 && (int64_t)s2 < (int64_t)s1 + l1;
}

static int contains(int32_t s_out, int32_t l_out, int32_t s_in, int32_t l_in)
{
    return s_out <= s_in && (int64_t)s_in + l_in <= (int64_t)s_out + l_out;
}

static int check_intervals(const int32_t* s, const int32_t* l, int32_t n)
{
    for (int32_t a = 0; a < n; a++)
        if (s[a] < 0 || l[a] < 1 || (int64_t)s[a] + l[a] > INT32_MAX) return -1;
    return 0;
}

int oracle_overlaps(const int32_t* arr_start, const int32_t* arr_len, int32_t n_arrays,
                    int64_t* ov_off, int32_t* ov_idx, int64_t ov_cap)
{
    if (n_arrays < 0 || check_intervals(arr_start, arr_len, n_arrays)) return -1;
    int64_t n = 0;
    ov_off[0] = 0;
    for (int32_t a = 0; a < n_arrays; a++) {
        for (int32_t b = 0; b < n_arrays; b++) {
            if (a == b || !overlap(arr_start[a], arr_len[a], arr_start[b], arr_len[b])) continue;
            if (n >= ov_cap) return -4;
            ov_idx[n++] = b;
        }
        ov_off[a + 1] = n;
    }
    return 0;
}

enum { M_R = 1, M_W = 2, M_RW = 3, M_DROPPED = 0x80 };

typedef struct {
    int32_t n_arrays;
    uint8_t* st;              /* 2A statuses: real 0..A-1, abstract A..2A-1 */
    int32_t* vff;
    int64_t ff;
    uint8_t* out_ks;
    int32_t* out_var;
    uint8_t* step;
    int64_t n, cap;
} vp_ctx;

/* Record one statement of the translated program and its effect on sigma. */
static int vp_emit(vp_ctx* c, int kind, int side, int32_t v, int after)
{
    if (c->n >= c->cap) return -4;      /* output capacity exceeded */
    int before = c->st[v];
    c->st[v] = (uint8_t)after;
    c->out_ks[c->n] = (uint8_t)(kind | side << 4);
    c->out_var[c->n] = v;
    c->step[c->n] = (uint8_t)after;
    if (after == ST_F && before != ST_F) {
        if (c->vff[v] < 0) c->vff[v] = (int32_t)c->n;
        if (c->ff < 0) c->ff = c->n;
    }
    c->n++;
    return 0;
}

static int vp_op(vp_ctx* c, int kind, int side, int32_t v)
{
    return vp_emit(c, kind, side, v, oracle_apply(kind, side, c->st[v]));
}

/* [[R x#]] and the guard part of [[RW x#]] (Fig. sem-AM):
 *   if (isValid x#) Noop else (Pull x; Pull x#)          -- CPU side
 *   if (remIsValid x#) Noop else (Push x; Push x#)       -- GPU side
 * Both statements are recorded (the GT and EN slots); when the condition holds
 * they leave their variable unchanged. */
static int vp_ensure(vp_ctx* c, int side, int32_t x)
{
    int32_t xa = c->n_arrays + x;
    int cond = is_valid_on(side, c->st[xa]);
    int rc = vp_emit(c, K_GT, side, x, cond ? c->st[x] : transfer_for(side, c->st[x]));
    if (rc) return rc;
    return vp_emit(c, K_EN, side, xa, cond ? c->st[xa] : transfer_for(side, c->st[xa]));
}

static int cmp_i32(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

int oracle_vectorpu(const int32_t* arr_start, const int32_t* arr_len, int32_t n_arrays,
                    const uint8_t* call_side, const int32_t* call_off, int64_t n_calls,
                    const int32_t* opnd_array, const uint8_t* opnd_mode, int infer_overlap,
                    uint8_t* out_kind_side, int32_t* out_var, int64_t out_cap, int64_t* out_n,
                    int64_t* call_first_op, uint8_t* step_status, uint8_t* final_status,
                    int32_t* var_first_fault, int64_t* first_fault)
{
    if (n_arrays < 0 || n_arrays > (INT32_MAX / 2) || n_calls < 0 || call_off[0] != 0) return -1;
    if (check_intervals(arr_start, arr_len, n_arrays)) return -1;
    for (int64_t c = 0; c < n_calls; c++) {
        if (call_off[c + 1] < call_off[c] || call_side[c] > 1) return -1;
        for (int32_t k = call_off[c]; k < call_off[c + 1]; k++) {
            uint8_t m = opnd_mode[k];
            if ((m & 0x7C) || (m & 3) == 0) return -1;
            if (opnd_array[k] < 0 || opnd_array[k] >= n_arrays) return -2;
            for (int32_t j = call_off[c]; j < k; j++)
                if (opnd_array[j] == opnd_array[k]) return -1;   /* footnote of Section 3.3 */
        }
    }
    /* r_v of Section 4.3: for every array, the arrays that overlap it (ascending) */
    int64_t* ov_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_arrays + 1));
    int64_t n_pairs = 0;
    for (int32_t a = 0; a < n_arrays; a++)
        for (int32_t b = 0; b < n_arrays; b++)
            n_pairs += (a != b && overlap(arr_start[a], arr_len[a], arr_start[b], arr_len[b]));
    int32_t* ov_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_pairs ? n_pairs : 1));
    int32_t nv = 2 * n_arrays;
    vp_ctx c;
    c.n_arrays = n_arrays;
    c.st = (uint8_t*)malloc((size_t)(nv ? nv : 1));
    c.vff = var_first_fault;
    c.ff = -1;
    c.out_ks = out_kind_side;
    c.out_var = out_var;
    c.step = step_status;
    c.n = 0;
    c.cap = out_cap;
    /* per-array scratch: mode in this call (0 = not an operand), effective
     * declared mode after O(M), shadow flag, and the list of shadows */
    uint8_t* opmode = (uint8_t*)calloc((size_t)(n_arrays ? n_arrays : 1), 1);
    uint8_t* eff = (uint8_t*)calloc((size_t)(n_arrays ? n_arrays : 1), 1);
    uint8_t* shadow = (uint8_t*)calloc((size_t)(n_arrays ? n_arrays : 1), 1);
    int32_t* shadow_list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_arrays ? n_arrays : 1));
    int rc = 0;
    if (!ov_off || !ov_idx || !c.st || !opmode || !eff || !shadow || !shadow_list) rc = -3;
    if (!rc) {
        int rc2 = oracle_overlaps(arr_start, arr_len, n_arrays, ov_off, ov_idx, n_pairs);
        if (rc2) rc = rc2;
    }
    for (int32_t v = 0; v < nv && !rc; v++) {
        c.st[v] = (uint8_t)encode((pair_t){ V, I });   /* real and abstract start at (V,I) */
        var_first_fault[v] = -1;
    }
    for (int64_t call = 0; call < n_calls && !rc; call++) {
        int side = call_side[call];
        int32_t k0 = call_off[call], k1 = call_off[call + 1];
        int32_t n_shadow = 0;
        call_first_op[call] = c.n;
        for (int32_t k = k0; k < k1; k++) {
            opmode[opnd_array[k]] = opnd_mode[k];
            eff[opnd_array[k]] = (opnd_mode[k] & M_DROPPED) ? 0 : (opnd_mode[k] & 3);
        }
        /* O(M), Table Overlap-ext-tab: the rules read the declared set M only
         * (not applied recursively, Section 4.3).  A dropped annotation is absent
         * from M and, being an argument of the call, is neither upgraded nor
         * shadowed. */
        if (infer_overlap) {
            for (int32_t k = k0; k < k1; k++) {
                int32_t x = opnd_array[k];
                uint8_t mx = opnd_mode[k];
                if ((mx & M_DROPPED) || !((mx & 3) & M_W)) continue;   /* x declared W or RW */
                for (int64_t j = ov_off[x]; j < ov_off[x + 1]; j++) {
                    int32_t y = ov_idx[j];
                    if (opmode[y] == 0) {
                        if (!shadow[y]) { shadow[y] = 1; shadow_list[n_shadow++] = y; }  /* RW y# */
                    } else if (!(opmode[y] & M_DROPPED)) {
                        /* RW rule: any y; W rule: only when W y# is not in M */
                        if ((mx & 3) == M_RW || (opmode[y] & 3) != M_W) eff[y] = M_RW;
                    }
                }
            }
            qsort(shadow_list, (size_t)n_shadow, sizeof(int32_t), cmp_i32);
        }
        /* [[O(M)]] then the body, grouped per operand in argument order (each
         * statement touches one variable, so per variable this is the paper's
         * order [[M]]; S) */
        for (int32_t k = k0; k < k1 && !rc; k++) {
            int32_t x = opnd_array[k];
            int mo = opnd_mode[k] & 3;
            if (!(opnd_mode[k] & M_DROPPED)) {
                int me = eff[x];
                if (me == M_R || me == M_RW) rc = vp_ensure(&c, side, x);
                if (!rc && (me == M_W || me == M_RW)) rc = vp_op(&c, K_W, side, n_arrays + x);
            }
            if (!rc && (mo == M_R || mo == M_RW)) rc = vp_op(&c, K_R, side, x);
            if (!rc && (mo == M_W || mo == M_RW)) rc = vp_op(&c, K_W, side, x);
        }
        /* shadow arguments RW(y), ascending array id (Section 4.3) */
        for (int32_t s = 0; s < n_shadow && !rc; s++) {
            int32_t y = shadow_list[s];
            rc = vp_ensure(&c, side, y);
            if (!rc) rc = vp_op(&c, K_W, side, n_arrays + y);
        }
        /* the body's writes also write the shared elements of overlapping arrays:
         * a wholly covered array is written, a partly covered one keeps its own
         * side and loses the other (the per-array summary reading) */
        for (int32_t k = k0; k < k1 && !rc; k++) {
            int32_t x = opnd_array[k];
            if (!((opnd_mode[k] & 3) & M_W)) continue;
            for (int64_t j = ov_off[x]; j < ov_off[x + 1] && !rc; j++) {
                int32_t y = ov_idx[j];
                int whole = contains(arr_start[x], arr_len[x], arr_start[y], arr_len[y]);
                rc = vp_op(&c, whole ? K_W : K_PW, side, y);
            }
        }
        for (int32_t k = k0; k < k1; k++) { opmode[opnd_array[k]] = 0; eff[opnd_array[k]] = 0; }
        for (int32_t s = 0; s < n_shadow; s++) shadow[shadow_list[s]] = 0;
    }
    if (!rc) {
        call_first_op[n_calls] = c.n;
        *out_n = c.n;
        for (int32_t v = 0; v < nv; v++) final_status[v] = c.st[v];
        *first_fault = c.ff;
    }
    free(ov_off);
    free(ov_idx);
    free(c.st);
    free(opmode);
    free(eff);
    free(shadow);
    free(shadow_list);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* VectorPU calls over pvectors that are created and deleted during the run  */
/* (Section 4.3: r_v is updated at pvector creations and deletions and       */
/* queried at calls; a partial vector inherits the coherence state of its    */
/* mother vector when it is declared, Section 5's description of VectorPU's  */
/* partial vectors).                                                          */
/*                                                                            */
/* r_v is kept as the paper's "simple unordered list": the live arrays, with */
/* every lookup a pass over all of them.  Array a is live at the calls       */
/* born[a] <= c < died[a].  parent[a] = -1 for a vector (its elements are a  */
/* fresh allocation: its statuses are those of the initial store), else the  */
/* vector whose range holds a's range and whose lifetime holds a's lifetime. */
/* Before call c, the pvectors born at c (ascending id) take their vector's  */
/* real and abstract statuses; the translated trace records each creation as */
/* Noop v, Noop v# (CPU side, no effect) at the head of call c's statements, */
/* and arr_probe[a] is the index of the first of the two (-1 for vectors).   */
/* The call's operands must be live; O(M), the shadows and the projections  */
/* of body writes range over the live arrays only.                           */
/* ------------------------------------------------------------------------ */
static int cmp_i64_first(const void* a, const void* b)
{
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

int oracle_vectorpu_lifetimes(const int32_t* arr_start, const int32_t* arr_len, const int32_t* arr_parent,
                              const int32_t* arr_born, const int32_t* arr_died, int32_t n_arrays,
                              const uint8_t* call_side, const int32_t* call_off, int64_t n_calls,
                              const int32_t* opnd_array, const uint8_t* opnd_mode, int infer_overlap,
                              uint8_t* out_kind_side, int32_t* out_var, int64_t out_cap, int64_t* out_n,
                              int64_t* call_first_op, int64_t* arr_probe, uint8_t* step_status,
                              uint8_t* final_status, int32_t* var_first_fault, int64_t* first_fault)
{
    if (n_arrays < 0 || n_arrays > (INT32_MAX / 2) || n_calls < 0 || n_calls > INT32_MAX || call_off[0] != 0)
        return -1;
    if (check_intervals(arr_start, arr_len, n_arrays)) return -1;
    for (int32_t a = 0; a < n_arrays; a++) {
        if (arr_born[a] < 0 || arr_born[a] >= arr_died[a] || arr_died[a] > n_calls) return -1;
        int32_t p = arr_parent[a];
        if (p == -1) continue;
        if (p < 0 || p >= n_arrays) return -2;
        if (p == a || arr_parent[p] != -1) return -1;                 /* a vector's own pvector */
        if (!contains(arr_start[p], arr_len[p], arr_start[a], arr_len[a])) return -1;
        if (arr_born[p] > arr_born[a] || arr_died[a] > arr_died[p]) return -1;
    }
    for (int64_t c = 0; c < n_calls; c++) {
        if (call_off[c + 1] < call_off[c] || call_side[c] > 1) return -1;
        for (int32_t k = call_off[c]; k < call_off[c + 1]; k++) {
            uint8_t m = opnd_mode[k];
            if ((m & 0x7C) || (m & 3) == 0) return -1;
            if (opnd_array[k] < 0 || opnd_array[k] >= n_arrays) return -2;
            int32_t x = opnd_array[k];
            if (c < arr_born[x] || c >= arr_died[x]) return -1;       /* not live at this call */
            for (int32_t j = call_off[c]; j < k; j++)
                if (opnd_array[j] == x) return -1;
        }
    }
    size_t An = (size_t)(n_arrays ? n_arrays : 1);
    int32_t nv = 2 * n_arrays;
    /* creation and deletion events ordered by call (then by id) */
    int64_t* births = (int64_t*)malloc(sizeof(int64_t) * An);
    int64_t* deaths = (int64_t*)malloc(sizeof(int64_t) * An);
    int32_t* live = (int32_t*)malloc(sizeof(int32_t) * An);       /* r_v: unordered */
    int32_t* live_pos = (int32_t*)malloc(sizeof(int32_t) * An);   /* index in live, -1 if dead */
    uint8_t* opmode = (uint8_t*)calloc(An, 1);
    uint8_t* eff = (uint8_t*)calloc(An, 1);
    uint8_t* shadow = (uint8_t*)calloc(An, 1);
    int32_t* list = (int32_t*)malloc(sizeof(int32_t) * An);
    vp_ctx c;
    c.n_arrays = n_arrays;
    c.st = (uint8_t*)malloc((size_t)(nv ? nv : 1));
    c.vff = var_first_fault;
    c.ff = -1;
    c.out_ks = out_kind_side;
    c.out_var = out_var;
    c.step = step_status;
    c.n = 0;
    c.cap = out_cap;
    int rc = 0;
    if (!births || !deaths || !live || !live_pos || !opmode || !eff || !shadow || !list || !c.st) rc = -3;
    int32_t n_live = 0;
    if (!rc) {
        for (int32_t a = 0; a < n_arrays; a++) {
            births[a] = ((int64_t)arr_born[a] << 32) | a;
            deaths[a] = ((int64_t)arr_died[a] << 32) | a;
            live_pos[a] = -1;
            arr_probe[a] = -1;
        }
        qsort(births, (size_t)n_arrays, sizeof(int64_t), cmp_i64_first);
        qsort(deaths, (size_t)n_arrays, sizeof(int64_t), cmp_i64_first);
        for (int32_t v = 0; v < nv; v++) {
            c.st[v] = (uint8_t)encode((pair_t){ V, I });   /* the initial store */
            var_first_fault[v] = -1;
        }
    }
    int32_t nb = 0, nd = 0;
    for (int64_t call = 0; call < n_calls && !rc; call++) {
        int side = call_side[call];
        int32_t k0 = call_off[call], k1 = call_off[call + 1];
        call_first_op[call] = c.n;
        /* deletions: arrays whose lifetime ended before this call leave r_v */
        while (nd < n_arrays && (deaths[nd] >> 32) <= call) {
            int32_t a = (int32_t)(deaths[nd] & 0xFFFFFFFF);
            int32_t i = live_pos[a];
            if (i >= 0) {
                live[i] = live[n_live - 1];
                live_pos[live[i]] = i;
                n_live--;
                live_pos[a] = -1;
            }
            nd++;
        }
        /* creations: join r_v; a pvector takes its vector's statuses */
        while (nb < n_arrays && (births[nb] >> 32) <= call && !rc) {
            int32_t a = (int32_t)(births[nb] & 0xFFFFFFFF);
            live_pos[a] = n_live;
            live[n_live++] = a;
            int32_t p = arr_parent[a];
            if (p >= 0) {
                arr_probe[a] = c.n;
                rc = vp_op(&c, K_NOOP, 0, p);
                if (!rc) rc = vp_op(&c, K_NOOP, 0, n_arrays + p);
                c.st[a] = c.st[p];
                c.st[n_arrays + a] = c.st[n_arrays + p];
            }
            nb++;
        }
        if (rc) break;
        for (int32_t k = k0; k < k1; k++) {
            opmode[opnd_array[k]] = opnd_mode[k];
            eff[opnd_array[k]] = (opnd_mode[k] & M_DROPPED) ? 0 : (opnd_mode[k] & 3);
        }
        int32_t n_shadow = 0;
        if (infer_overlap) {
            /* O(M) against the live arrays, Table Overlap-ext-tab (declared set
             * only, not applied again to what it adds) */
            for (int32_t k = k0; k < k1; k++) {
                int32_t x = opnd_array[k];
                uint8_t mx = opnd_mode[k];
                if ((mx & M_DROPPED) || !((mx & 3) & M_W)) continue;
                for (int32_t i = 0; i < n_live; i++) {
                    int32_t y = live[i];
                    if (y == x || !overlap(arr_start[x], arr_len[x], arr_start[y], arr_len[y])) continue;
                    if (opmode[y] == 0) {
                        if (!shadow[y]) { shadow[y] = 1; list[n_shadow++] = y; }
                    } else if (!(opmode[y] & M_DROPPED)) {
                        if ((mx & 3) == M_RW || (opmode[y] & 3) != M_W) eff[y] = M_RW;
                    }
                }
            }
            qsort(list, (size_t)n_shadow, sizeof(int32_t), cmp_i32);
        }
        for (int32_t k = k0; k < k1 && !rc; k++) {
            int32_t x = opnd_array[k];
            int mo = opnd_mode[k] & 3;
            if (!(opnd_mode[k] & M_DROPPED)) {
                int me = eff[x];
                if (me == M_R || me == M_RW) rc = vp_ensure(&c, side, x);
                if (!rc && (me == M_W || me == M_RW)) rc = vp_op(&c, K_W, side, n_arrays + x);
            }
            if (!rc && (mo == M_R || mo == M_RW)) rc = vp_op(&c, K_R, side, x);
            if (!rc && (mo == M_W || mo == M_RW)) rc = vp_op(&c, K_W, side, x);
        }
        for (int32_t s2 = 0; s2 < n_shadow && !rc; s2++) {
            int32_t y = list[s2];
            rc = vp_ensure(&c, side, y);
            if (!rc) rc = vp_op(&c, K_W, side, n_arrays + y);
        }
        for (int32_t s2 = 0; s2 < n_shadow; s2++) shadow[list[s2]] = 0;
        /* the body's writes reach the shared elements of the live arrays that
         * overlap the operand, in ascending id */
        for (int32_t k = k0; k < k1 && !rc; k++) {
            int32_t x = opnd_array[k];
            if (!((opnd_mode[k] & 3) & M_W)) continue;
            int32_t n_ov = 0;
            for (int32_t i = 0; i < n_live; i++) {
                int32_t y = live[i];
                if (y != x && overlap(arr_start[x], arr_len[x], arr_start[y], arr_len[y])) list[n_ov++] = y;
            }
            qsort(list, (size_t)n_ov, sizeof(int32_t), cmp_i32);
            for (int32_t j = 0; j < n_ov && !rc; j++) {
                int32_t y = list[j];
                int whole = contains(arr_start[x], arr_len[x], arr_start[y], arr_len[y]);
                rc = vp_op(&c, whole ? K_W : K_PW, side, y);
            }
        }
        for (int32_t k = k0; k < k1; k++) { opmode[opnd_array[k]] = 0; eff[opnd_array[k]] = 0; }
    }
    if (!rc) {
        call_first_op[n_calls] = c.n;
        *out_n = c.n;
        for (int32_t v = 0; v < nv; v++) final_status[v] = c.st[v];
        *first_fault = c.ff;
    }
    free(births);
    free(deaths);
    free(live);
    free(live_pos);
    free(opmode);
    free(eff);
    free(shadow);
    free(list);
    free(c.st);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Static well-declaredness (Section 3.3: Definitions "Occurs in all         */
/* execution paths" and "Well-declared program"; Section 3.5: Definition     */
/* "Well-declared program with array access").                               */
/* ------------------------------------------------------------------------ */

/* Whether the op "w on side `side` of location loc" occurs in all execution
 * paths of the statement sequence [lo, hi).  Conditions are opaque, so every
 * branch of an If and every iteration count of a While (zero included) is a
 * path: a sequence has the op on all paths when one of its items has; an op
 * item when it is that op; an If when both branches have; a While never (its
 * body may run zero times).  Returns 1 / 0, or -1 on malformed tokens. */
static int wd_must_write(const uint8_t* tok, const int32_t* payload, int64_t lo, int64_t hi,
                         int32_t loc, int side, int depth)
{
    if (depth > ORACLE_MAX_DEPTH) return -1;
    int found = 0;
    int64_t i = lo;
    while (i < hi) {
        int k = tok[i] & 15, sd = (tok[i] >> 4) & 1;
        if (k <= K_NOOP) {
            if (k == K_W && sd == side && payload[i] == loc) found = 1;
            i++;
        } else if (k == T_IF) {
            int64_t e = i + 1 + payload[i];
            if (payload[i] < 0 || e >= hi || tok[e] != T_ELSE || sd) return -1;
            int64_t end = e + 1 + payload[e];
            if (payload[e] < 0 || end >= hi || tok[end] != T_END) return -1;
            int a = wd_must_write(tok, payload, i + 1, e, loc, side, depth + 1);
            int b = wd_must_write(tok, payload, e + 1, end, loc, side, depth + 1);
            if (a < 0 || b < 0) return -1;
            if (a && b) found = 1;
            i = end + 1;
        } else if (k == T_WHILE) {
            int64_t end = i + 1 + payload[i];
            if (payload[i] < 0 || end >= hi || tok[end] != T_END || sd) return -1;
            int a = wd_must_write(tok, payload, i + 1, end, loc, side, depth + 1);   /* validates the body */
            if (a < 0) return -1;
            i = end + 1;
        } else {
            return -1;
        }
    }
    return found;
}

int oracle_well_declared(const int64_t* arr_loc_off, int32_t n_arrays, const int32_t* loc_owner,
                         const int64_t* call_tok_off, int64_t n_calls, const uint8_t* tok,
                         const int32_t* payload, const int64_t* call_am_off, const int32_t* am_array,
                         const uint8_t* am_mode, uint32_t* violations, int64_t* first_bad,
                         int32_t* first_unmet)
{
    if (n_arrays < 0 || n_calls < 0) return -1;
    const int64_t n_locs = arr_loc_off[n_arrays];
    for (int32_t a = 0; a < n_arrays; a++) {
        if (arr_loc_off[a + 1] < arr_loc_off[a]) return -1;
        for (int64_t l = arr_loc_off[a]; l < arr_loc_off[a + 1]; l++)
            if (loc_owner[l] != a) return -1;
    }
    for (int64_t c = 0; c < n_calls; c++) {
        const int64_t t0 = call_tok_off[c], t1 = call_tok_off[c + 1];
        const int64_t m0 = call_am_off[c], m1 = call_am_off[c + 1];
        if (t1 < t0 || m1 < m0) return -1;
        uint32_t viol = 0;
        int64_t bad = -1;
        int32_t unmet = -1;
        if (wd_must_write(tok, payload, t0, t1, -1, 0, 0) < 0) return -1;   /* structure well formed */
        /* the declarations: an array may appear once (Section 3.3, syntax of AM) */
        for (int64_t j = m0; j < m1; j++) {
            if (am_array[j] < 0 || am_array[j] >= n_arrays) return -2;
            int md = am_mode[j] & 15;
            if ((am_mode[j] & 0xE0) || md < 1 || md > 3) return -1;
            for (int64_t j2 = m0; j2 < j; j2++)
                if (am_array[j2] == am_array[j]) viol |= 16u;
        }
        /* every statement of the body against the declarations */
        for (int64_t i = t0; i < t1; i++) {
            int k = tok[i] & 15, sd = (tok[i] >> 4) & 1;
            if (tok[i] & 0xE0) return -1;
            if (k > K_NOOP) {
                if (k == K_PW || k == K_GT || k == K_EN) return -1;   /* not statements of a body */
                continue;                                           /* structure tokens */
            }
            if (k == K_NOOP) continue;
            if (payload[i] < 0 || payload[i] >= n_locs) return -2;
            uint32_t v = 0;
            if (k == K_PUSH || k == K_PULL) {
                v = 1u;                                   /* no Push / Pull in a function body */
            } else {
                const int32_t a = loc_owner[payload[i]];
                int ok = 0;
                for (int64_t j = m0; j < m1; j++) {
                    if (am_array[j] != a || ((am_mode[j] >> 4) & 1) != sd) continue;
                    int md = am_mode[j] & 15;
                    if (k == K_W && (md == 2 || md == 3)) ok = 1;       /* W or RW */
                    if (k == K_R && (md == 1 || md == 3)) ok = 1;       /* R or RW */
                }
                if (!ok) v = k == K_W ? 2u : 4u;
            }
            if (v) {
                viol |= v;
                if (bad < 0) bad = i - t0;
            }
        }
        /* W obligations: every location of the array written, on the declared
         * side, in all execution paths of the body */
        for (int64_t j = m0; j < m1; j++) {
            if ((am_mode[j] & 15) != 2) continue;
            const int32_t a = am_array[j];
            const int side = (am_mode[j] >> 4) & 1;
            for (int64_t l = arr_loc_off[a]; l < arr_loc_off[a + 1]; l++) {
                int r = wd_must_write(tok, payload, t0, t1, (int32_t)l, side, 0);
                if (r < 0) return -1;
                if (!r) {
                    viol |= 8u;
                    if (unmet < 0 || a < unmet) unmet = a;
                    break;
                }
            }
        }
        violations[c] = viol;
        first_bad[c] = bad;
        first_unmet[c] = unmet;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* More than two memory locations (Section 3 states the results extend to    */
/* many locations; the conclusion names it as future work).  The status of a */
/* variable is a vector of k validity flags (location 0 = main memory, where */
/* data starts, Section 3.2).  Each op runs at a location; the Section 3.1    */
/* signatures, written for a vector instead of a pair:                       */
/*   r at a:           flag a must be V; nothing changes                     */
/*   w at a:           flag a becomes V, every other flag I                  */
/*   copy a -> b:      flag a must be V; flag b becomes V (Push at a towards */
/*                     b, or Pull at b from a; with k = 2, local 0 and       */
/*                     remote 1: Push = copy 0->1, Pull = copy 1->0,         */
/*                     rem Push = copy 1->0, rem Pull = copy 0->1)           */
/*   Noop:             nothing changes                                       */
/* A requirement that fails leaves the variable stuck (F), as in Property    */
/* Progress.  Op byte: bits 0-1 kind (r 0, w 1, copy 2, Noop 3), bits 2-4   */
/* location a, bits 5-7 location b (copy only; 0 otherwise, and a = 0 for    */
/* Noop).  Status byte: bit i = flag of location i is V; F = 0x80; k <= 7.   */
/* ------------------------------------------------------------------------ */
enum { KL_R = 0, KL_W = 1, KL_COPY = 2, KL_NOOP = 3, KL_F = 0x80, KL_MAX = 7 };

typedef struct { int valid[KL_MAX]; } kvec_t;

static int kl_valid_byte(uint8_t op, int k)
{
    int kind = op & 3, a = (op >> 2) & 7, b = (op >> 5) & 7;
    if (kind == KL_NOOP) return a == 0 && b == 0;
    if (a >= k) return 0;
    if (kind == KL_COPY) return b < k && b != a;
    return b == 0;
}

/* status byte of applying op to status byte s (k locations) */
int oracle_apply_k(int op, int s, int k)
{
    if (k < 1 || k > KL_MAX || !kl_valid_byte((uint8_t)op, k)) return -1;
    if (s & KL_F) return KL_F;
    kvec_t v = {{0}};
    for (int i = 0; i < k; i++) v.valid[i] = (s >> i) & 1;
    int kind = op & 3, a = (op >> 2) & 7, b = (op >> 5) & 7;
    switch (kind) {
    case KL_R:                                     /* (.., V_a, ..) -> same */
        if (!v.valid[a]) return KL_F;
        break;
    case KL_W:                                     /* any -> V at a only */
        for (int i = 0; i < k; i++) v.valid[i] = (i == a);
        break;
    case KL_COPY:                                  /* (.., V_a, ..) -> (.., V_b, ..) */
        if (!v.valid[a]) return KL_F;
        v.valid[b] = 1;
        break;
    default:                                       /* Noop */
        break;
    }
    int out = 0;
    for (int i = 0; i < k; i++) out |= v.valid[i] << i;
    return out;
}

int oracle_check_trace_k(const uint8_t* op, const int32_t* var, int64_t n_ops, int32_t n_vars, int32_t k,
                         const uint8_t* init_status, uint8_t* step_status, uint8_t* final_status,
                         int32_t* var_first_fault, int64_t* first_fault)
{
    if (n_ops < 0 || n_vars < 0 || k < 1 || k > KL_MAX) return -1;
    for (int64_t i = 0; i < n_ops; i++) {
        if (!kl_valid_byte(op[i], k)) return -1;
        if (var[i] < 0 || var[i] >= n_vars) return -2;
    }
    uint8_t* st = (uint8_t*)malloc((size_t)(n_vars ? n_vars : 1));
    if (!st) return -3;
    for (int32_t v = 0; v < n_vars; v++) {
        st[v] = init_status ? init_status[v] : (uint8_t)1;       /* valid in location 0 only */
        if (st[v] != KL_F && (st[v] >> k)) { free(st); return -1; }
        var_first_fault[v] = -1;
    }
    int64_t ff = -1;
    for (int64_t i = 0; i < n_ops; i++) {
        int v = var[i], before = st[v], after = oracle_apply_k(op[i], before, k);
        st[v] = (uint8_t)after;
        step_status[i] = (uint8_t)after;
        if (after == KL_F && before != KL_F) {
            if (var_first_fault[v] < 0) var_first_fault[v] = (int32_t)i;
            if (ff < 0) ff = i;
        }
    }
    for (int32_t v = 0; v < n_vars; v++) final_status[v] = st[v];
    *first_fault = ff;
    free(st);
    return 0;
}
