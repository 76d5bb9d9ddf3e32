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
