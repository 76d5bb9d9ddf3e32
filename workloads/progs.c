/*
 * progs.c -- seeded generator of synthetic structured programs (token streams
 * with If/While nesting).  Input generation only: it holds none of the checked
 * calculus' arithmetic and is shared by the oracle tests and the GPU path.
 *
 * Random numbers: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), one stream
 * per program seeded from (seed, program index), so programs can be generated
 * independently and the size pass and the fill pass agree.
 *
 * Token layout: op byte (kind | side << 4) and int32 payload.  Ops carry their
 * program-local variable id; IF / ELSE / WHILE carry the token length of the
 * branch or body that follows; END carries 0.
 *   IF(len_then) <then> ELSE(len_else) <else> END
 *   WHILE(len_body) <body> END
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s; } rng_t;

static uint64_t next_u64(rng_t* r)
{
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double u01(rng_t* r) { return (double)(next_u64(r) >> 11) * (1.0 / 9007199254740992.0); }
static int64_t uniform_int(rng_t* r, int64_t lo, int64_t hi)   /* inclusive */
{
    return lo + (int64_t)(u01(r) * (double)(hi - lo + 1));
}
static double normal(rng_t* r)                                 /* Box-Muller */
{
    double u1 = u01(r), u2 = u01(r);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

typedef struct {
    double p_if, p_while;
    int max_depth, max_branch, max_body;
    double median, sigma;
    int64_t max_len;
    int vars_lo, vars_hi;
    double kind_cdf[5];            /* r, w, Push, Pull, Noop */
} prog_params;

typedef struct {
    rng_t rng;
    const prog_params* pp;
    int32_t n_vars;
    uint8_t* tok;                  /* NULL in the size pass */
    int32_t* payload;
    int64_t n;
} gen_ctx;

static void put(gen_ctx* g, uint8_t t, int32_t p)
{
    if (g->tok) { g->tok[g->n] = t; g->payload[g->n] = p; }
    g->n++;
}

static void gen_seq(gen_ctx* g, int64_t budget, int depth)
{
    const prog_params* pp = g->pp;
    while (budget > 0) {
        double u = u01(&g->rng);
        if (depth < pp->max_depth && u < pp->p_if) {
            int64_t t = uniform_int(&g->rng, 0, pp->max_branch);
            int64_t e = uniform_int(&g->rng, 0, pp->max_branch);
            if (t > budget) t = budget;
            if (e > budget - t) e = budget - t;
            int64_t at_if = g->n;
            put(g, 8, 0);
            gen_seq(g, t, depth + 1);
            int64_t at_else = g->n;
            put(g, 9, 0);
            gen_seq(g, e, depth + 1);
            if (g->tok) {
                g->payload[at_if] = (int32_t)(at_else - at_if - 1);
                g->payload[at_else] = (int32_t)(g->n - at_else - 1);
            }
            put(g, 11, 0);
            budget -= t + e;
        } else if (depth < pp->max_depth && u < pp->p_if + pp->p_while) {
            int64_t b = uniform_int(&g->rng, 1, pp->max_body);
            if (b > budget) b = budget;
            int64_t at_w = g->n;
            put(g, 10, 0);
            gen_seq(g, b, depth + 1);
            if (g->tok) g->payload[at_w] = (int32_t)(g->n - at_w - 1);
            put(g, 11, 0);
            budget -= b;
        } else {
            double k = u01(&g->rng);
            int kind = 0;
            while (kind < 4 && k >= pp->kind_cdf[kind]) kind++;
            int side = (int)(next_u64(&g->rng) >> 63);
            int32_t v = (int32_t)uniform_int(&g->rng, 0, g->n_vars - 1);
            put(g, (uint8_t)(kind | side << 4), v);
            budget--;
        }
    }
}

static void gen_program(const prog_params* pp, uint64_t seed, int64_t index,
                        uint8_t* tok, int32_t* payload, int64_t* n_tok, int32_t* n_vars,
                        int64_t* n_leaf)
{
    gen_ctx g;
    g.rng.s = seed * 0x2545F4914F6CDD1Dull + (uint64_t)index * 0x9E3779B97F4A7C15ull + 1;
    next_u64(&g.rng);
    g.pp = pp;
    g.n_vars = (int32_t)uniform_int(&g.rng, pp->vars_lo, pp->vars_hi);
    double len = floor(exp(log(pp->median) + pp->sigma * normal(&g.rng)) + 0.5);
    if (len < 1) len = 1;
    if (len > (double)pp->max_len) len = (double)pp->max_len;
    g.tok = tok;
    g.payload = payload;
    g.n = 0;
    gen_seq(&g, (int64_t)len, 0);
    *n_tok = g.n;
    *n_vars = g.n_vars;
    *n_leaf = (int64_t)len;
}

/* params: p_if, p_while, median, sigma, kind_cdf[5]; iparams: max_depth,
 * max_branch, max_body, max_len, vars_lo, vars_hi */
static void unpack(prog_params* pp, const double* params, const int64_t* iparams)
{
    pp->p_if = params[0];
    pp->p_while = params[1];
    pp->median = params[2];
    pp->sigma = params[3];
    for (int k = 0; k < 5; k++) pp->kind_cdf[k] = params[4 + k];
    pp->max_depth = (int)iparams[0];
    pp->max_branch = (int)iparams[1];
    pp->max_body = (int)iparams[2];
    pp->max_len = iparams[3];
    pp->vars_lo = (int)iparams[4];
    pp->vars_hi = (int)iparams[5];
}

/* Size pass: token count, variable count and leaf-op count of programs
 * [first, first + n). */
void wl_program_sizes(const double* params, const int64_t* iparams, uint64_t seed,
                      int64_t first, int64_t n, int64_t* n_tok, int32_t* n_vars, int64_t* n_leaf)
{
    prog_params pp;
    unpack(&pp, params, iparams);
    for (int64_t p = 0; p < n; p++)
        gen_program(&pp, seed, first + p, NULL, NULL, &n_tok[p], &n_vars[p], &n_leaf[p]);
}

/* Fill pass: writes program p's tokens at tok_off[p] (relative offsets). */
void wl_program_fill(const double* params, const int64_t* iparams, uint64_t seed,
                     int64_t first, int64_t n, const int64_t* tok_off,
                     uint8_t* tok, int32_t* payload)
{
    prog_params pp;
    unpack(&pp, params, iparams);
    for (int64_t p = 0; p < n; p++) {
        int64_t nt, nl;
        int32_t nv;
        gen_program(&pp, seed, first + p, tok + tok_off[p], payload + tok_off[p], &nt, &nv, &nl);
    }
}

/* ------------------------------------------------------------------------ */
/* Calls AM{S} for the static well-declaredness check: declarations over     */
/* arrays of locations and a structured body built from them.               */
/*   arrays: a owns locations [a_off[a], a_off[a+1]) (given by the caller)   */
/*   per call (own SplitMix64 stream from (seed, call index)): one side; 1..4 */
/*   declarations on distinct arrays, modes R / W / RW with p_mode[];        */
/*   body items in a random order: for W, every location written, at top    */
/*   level, or in both branches of an If; for R, 1..4 reads; for RW, reads   */
/*   and writes; a Noop now and then.  With probability p_bad the call gets  */
/*   one injected flaw: a W array written in one branch only, or inside a    */
/*   While; a read or write of an undeclared array; a read of a W array; a   */
/*   Push.                                                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    rng_t rng;
    uint8_t* tok;
    int32_t* payload;
    int64_t n;
} wd_ctx;

static void wput(wd_ctx* g, uint8_t t, int32_t p)
{
    if (g->tok) {
        g->tok[g->n] = t;
        g->payload[g->n] = p;
    }
    g->n++;
}

/* writes of every location of array a, in order */
static void wd_write_all(wd_ctx* g, const int64_t* a_off, int32_t a, int side)
{
    for (int64_t l = a_off[a]; l < a_off[a + 1]; l++) wput(g, (uint8_t)(1 | side << 4), (int32_t)l);
}

static int64_t wd_call(wd_ctx* g, const int64_t* a_off, int32_t n_arrays, const double* p_mode, double p_bad,
                       int32_t* am_array, uint8_t* am_mode)
{
    const int side = (int)uniform_int(&g->rng, 0, 1);
    int nd = (int)uniform_int(&g->rng, 1, 4);
    if (nd > n_arrays) nd = n_arrays;
    int32_t arr[4];
    int mode[4];
    for (int i = 0; i < nd; i++) {
        int32_t a;
        int dup;
        do {
            a = (int32_t)uniform_int(&g->rng, 0, n_arrays - 1);
            dup = 0;
            for (int j = 0; j < i; j++) dup |= arr[j] == a;
        } while (dup);
        arr[i] = a;
        double u = u01(&g->rng);
        mode[i] = u < p_mode[0] ? 1 : (u < p_mode[0] + p_mode[1] ? 2 : 3);
        if (am_array) {
            am_array[i] = a;
            am_mode[i] = (uint8_t)(mode[i] | side << 4);
        }
    }
    const int bad = u01(&g->rng) < p_bad ? (int)uniform_int(&g->rng, 1, 5) : 0;
    const int victim = (int)uniform_int(&g->rng, 0, nd - 1);
    /* items in a random order: a permutation of the declarations */
    int order[4] = {0, 1, 2, 3};
    for (int i = nd - 1; i > 0; i--) {
        int j = (int)uniform_int(&g->rng, 0, i);
        int t = order[i];
        order[i] = order[j];
        order[j] = t;
    }
    for (int oi = 0; oi < nd; oi++) {
        const int i = order[oi];
        const int32_t a = arr[i];
        const int64_t len = a_off[a + 1] - a_off[a];
        if (mode[i] == 2) {
            if (bad == 1 && i == victim) {               /* written in one branch only */
                int64_t at = g->n;
                wput(g, 8, 0);
                int64_t b0 = g->n;
                wd_write_all(g, a_off, a, side);
                if (g->tok) g->payload[at] = (int32_t)(g->n - b0);
                wput(g, 9, 1);
                wput(g, (uint8_t)(4 | side << 4), (int32_t)a_off[a]);
                wput(g, 11, 0);
            } else if (bad == 2 && i == victim) {        /* written inside a While only */
                int64_t at = g->n;
                wput(g, 10, 0);
                int64_t b0 = g->n;
                wd_write_all(g, a_off, a, side);
                if (g->tok) g->payload[at] = (int32_t)(g->n - b0);
                wput(g, 11, 0);
            } else if (u01(&g->rng) < 0.3) {             /* both branches write every location */
                int64_t at = g->n;
                wput(g, 8, 0);
                int64_t b0 = g->n;
                wd_write_all(g, a_off, a, side);
                if (g->tok) g->payload[at] = (int32_t)(g->n - b0);
                int64_t at2 = g->n;
                wput(g, 9, 0);
                int64_t b1 = g->n;
                wd_write_all(g, a_off, a, side);
                if (g->tok) g->payload[at2] = (int32_t)(g->n - b1);
                wput(g, 11, 0);
            } else {
                wd_write_all(g, a_off, a, side);
            }
            if (bad == 3 && i == victim) wput(g, (uint8_t)(0 | side << 4), (int32_t)a_off[a]);   /* read under W */
        } else {
            const int nr = (int)uniform_int(&g->rng, 1, 4);
            const int in_while = u01(&g->rng) < 0.2;
            int64_t at = g->n;
            if (in_while) wput(g, 10, 0);
            int64_t b0 = g->n;
            for (int r = 0; r < nr; r++) {
                const int32_t l = (int32_t)(a_off[a] + uniform_int(&g->rng, 0, len - 1));
                wput(g, (uint8_t)(0 | side << 4), l);
                if (mode[i] == 3 && u01(&g->rng) < 0.5) wput(g, (uint8_t)(1 | side << 4), l);
            }
            if (in_while) {
                if (g->tok) g->payload[at] = (int32_t)(g->n - b0);
                wput(g, 11, 0);
            }
        }
        if (u01(&g->rng) < 0.2) wput(g, (uint8_t)(4 | side << 4), (int32_t)a_off[a]);
    }
    if (bad == 4) {                                      /* an access to an undeclared array */
        int32_t a;
        int dup;
        int tries = 0;
        do {
            a = (int32_t)uniform_int(&g->rng, 0, n_arrays - 1);
            dup = 0;
            for (int j = 0; j < nd; j++) dup |= arr[j] == a;
        } while (dup && ++tries < 8);
        wput(g, (uint8_t)((int)uniform_int(&g->rng, 0, 1) | side << 4), (int32_t)a_off[a]);
    } else if (bad == 5) {
        wput(g, (uint8_t)(2 | side << 4), (int32_t)a_off[arr[victim]]);          /* Push in a body */
    }
    return nd;
}

/* size pass: tokens and declarations per call */
void wl_wd_sizes(const int64_t* a_off, int32_t n_arrays, uint64_t seed, int64_t n_calls, const double* p_mode,
                 double p_bad, int64_t* n_tok, int32_t* n_decl)
{
    for (int64_t c = 0; c < n_calls; c++) {
        wd_ctx g = {{seed * 0x9E3779B97F4A7C15ull + (uint64_t)c * 0xD1B54A32D192ED03ull}, NULL, NULL, 0};
        n_decl[c] = (int32_t)wd_call(&g, a_off, n_arrays, p_mode, p_bad, NULL, NULL);
        n_tok[c] = g.n;
    }
}

/* fill pass, into CSR offsets computed from the size pass */
void wl_wd_fill(const int64_t* a_off, int32_t n_arrays, uint64_t seed, int64_t n_calls, const double* p_mode,
                double p_bad, const int64_t* tok_off, const int64_t* am_off, uint8_t* tok, int32_t* payload,
                int32_t* am_array, uint8_t* am_mode)
{
    for (int64_t c = 0; c < n_calls; c++) {
        wd_ctx g = {{seed * 0x9E3779B97F4A7C15ull + (uint64_t)c * 0xD1B54A32D192ED03ull}, tok + tok_off[c],
                    payload + tok_off[c], 0};
        wd_call(&g, a_off, n_arrays, p_mode, p_bad, am_array + am_off[c], am_mode + am_off[c]);
    }
}

/* ------------------------------------------------------------------------ */
/* VectorPU calls over pvectors with lifetimes.  Arrays [0, n_vectors) are   */
/* vectors (parent -1, live for the whole run); the rest are pvectors of a   */
/* uniformly drawn vector: a sub-range of it (start uniform in the vector,   */
/* length floor(2^U(len_lo, len_hi)) clipped to the vector's end), created   */
/* before a uniformly drawn call and deleted after floor(mean_life * E) more */
/* calls (E exponential, at least one call, clipped to the run).  Each call  */
/* has a fair side and 1..max_opnds distinct operands drawn uniformly from   */
/* the arrays live at that call (creations and deletions happen between      */
/* calls), modes R / W / RW with p_mode and annotations dropped with p_drop. */
/* One stream for the arrays and one for the calls, both SplitMix64.         */
/* ------------------------------------------------------------------------ */
static void wl_sort_events(int64_t* ev, int32_t n)                /* ascending, heap sort */
{
    for (int32_t i = n / 2 - 1; i >= 0; i--) {
        for (int32_t r = i;;) {
            int32_t c = 2 * r + 1;
            if (c >= n) break;
            if (c + 1 < n && ev[c + 1] > ev[c]) c++;
            if (ev[r] >= ev[c]) break;
            int64_t t = ev[r]; ev[r] = ev[c]; ev[c] = t; r = c;
        }
    }
    for (int32_t e = n - 1; e > 0; e--) {
        int64_t t = ev[0]; ev[0] = ev[e]; ev[e] = t;
        for (int32_t r = 0;;) {
            int32_t c = 2 * r + 1;
            if (c >= e) break;
            if (c + 1 < e && ev[c + 1] > ev[c]) c++;
            if (ev[r] >= ev[c]) break;
            t = ev[r]; ev[r] = ev[c]; ev[c] = t; r = c;
        }
    }
}

void wl_lifetimes_arrays(uint64_t seed, int32_t n_vectors, int32_t vec_len, int32_t n_arrays, int64_t n_calls,
                         double len_lo, double len_hi, double mean_life, int32_t* start, int32_t* len,
                         int32_t* parent, int32_t* born, int32_t* died)
{
    rng_t r = {seed * 0x9E3779B97F4A7C15ull + 0x5851F42D4C957F2Dull};
    for (int32_t a = 0; a < n_arrays; a++) {
        if (a < n_vectors) {
            start[a] = a * vec_len;
            len[a] = vec_len;
            parent[a] = -1;
            born[a] = 0;
            died[a] = (int32_t)n_calls;
            continue;
        }
        int32_t v = (int32_t)uniform_int(&r, 0, n_vectors - 1);
        int32_t off = (int32_t)uniform_int(&r, 0, vec_len - 1);
        double l = floor(pow(2.0, len_lo + (len_hi - len_lo) * u01(&r)));
        int64_t ln = (int64_t)l < 1 ? 1 : (int64_t)l;
        if (ln > vec_len - off) ln = vec_len - off;
        start[a] = v * vec_len + off;
        len[a] = (int32_t)ln;
        parent[a] = v;
        int64_t b = uniform_int(&r, 0, n_calls - 1);
        double u = u01(&r);
        int64_t life = (int64_t)floor(-mean_life * log(u < 1e-300 ? 1e-300 : u));
        if (life < 1) life = 1;
        int64_t d = b + life > n_calls ? n_calls : b + life;
        born[a] = (int32_t)b;
        died[a] = (int32_t)d;
    }
}

/* calls; counts[c] = operands of call c when opnd_array is NULL (size pass),
 * else the operands are written at call_off[c] */
int wl_lifetimes_calls(uint64_t seed, int32_t n_arrays, const int32_t* born, const int32_t* died, int64_t n_calls,
                       int32_t max_opnds, const double* p_mode, double p_drop, uint8_t* side, int32_t* counts,
                       const int64_t* call_off, int32_t* opnd_array, uint8_t* opnd_mode)
{
    rng_t r = {seed * 0xD1B54A32D192ED03ull + 0x2545F4914F6CDD1Dull};
    int64_t* births = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_arrays ? n_arrays : 1));
    int64_t* deaths = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_arrays ? n_arrays : 1));
    int32_t* live = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_arrays ? n_arrays : 1));
    int32_t* pos = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_arrays ? n_arrays : 1));
    if (!births || !deaths || !live || !pos) {
        free(births); free(deaths); free(live); free(pos);
        return -3;
    }
    for (int32_t a = 0; a < n_arrays; a++) {
        births[a] = ((int64_t)born[a] << 32) | a;
        deaths[a] = ((int64_t)died[a] << 32) | a;
        pos[a] = -1;
    }
    wl_sort_events(births, n_arrays);
    wl_sort_events(deaths, n_arrays);
    int32_t n_live = 0, nb = 0, nd = 0;
    int32_t pick[64];
    for (int64_t c = 0; c < n_calls; c++) {
        while (nd < n_arrays && (deaths[nd] >> 32) <= c) {
            int32_t a = (int32_t)(deaths[nd++] & 0xFFFFFFFF);
            int32_t i = pos[a];
            if (i >= 0) { live[i] = live[--n_live]; pos[live[i]] = i; pos[a] = -1; }
        }
        while (nb < n_arrays && (births[nb] >> 32) <= c) {
            int32_t a = (int32_t)(births[nb++] & 0xFFFFFFFF);
            pos[a] = n_live;
            live[n_live++] = a;
        }
        side[c] = (uint8_t)(next_u64(&r) & 1);
        int32_t k = (int32_t)uniform_int(&r, 1, max_opnds);
        if (k > n_live) k = n_live;
        if (k > 64) k = 64;
        for (int32_t j = 0; j < k; j++) {
            int32_t a, dup;
            do {
                a = live[uniform_int(&r, 0, n_live - 1)];
                dup = 0;
                for (int32_t i = 0; i < j; i++) dup |= pick[i] == a;
            } while (dup);
            pick[j] = a;
            double u = u01(&r);
            uint8_t m = u < p_mode[0] ? 1 : (u < p_mode[0] + p_mode[1] ? 2 : 3);
            if (u01(&r) < p_drop) m |= 0x80;
            if (opnd_array) {
                opnd_array[call_off[c] + j] = a;
                opnd_mode[call_off[c] + j] = m;
            }
        }
        counts[c] = k;
    }
    free(births); free(deaths); free(live); free(pos);
    return 0;
}
