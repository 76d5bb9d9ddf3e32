// monoid.cu -- transfer functions of single ops and the finite monoid they
// generate under sequential composition; the device error word.
//
// Each op acts on one variable's status (Section 3.1 signatures, Fig. Opsem
// rules Effect / Remote Effect).  Written per side: "own" is the flag of the
// memory the op runs on (CPU for E x, GPU for rem(E x)), "other" the flag of
// the other memory.
//   r    needs own valid; no change
//   w    own := V, other := I
//   Push needs own valid; other := V
//   Pull needs other valid; own := V        (Pull = rem Push, Section 3.2)
//   Noop no change
//   pw   other := I                          (partial write of an overlapping array)
//   EN   own valid: no change; else the transfer of Fig. sem-AM (needs other
//        valid; own := V)
// A failed need gives the stuck status F, which every op keeps.  The closure
// of these 14 functions under composition has 32 elements; elements are
// numbered in discovery order with the identity first.
#include <map>
#include <mutex>
#include <vector>

#include "amc_internal.cuh"

namespace amc {

__device__ int g_error_word;

namespace {

using Map = std::vector<uint8_t>;   // status 0..4 -> status 0..4

int own_bit(int side) { return side == 0 ? 1 : 2; }
int other_bit(int side) { return side == 0 ? 2 : 1; }

int step(int kind, int side, int s)
{
    if (s == ST_F) return ST_F;
    const int own = own_bit(side), other = other_bit(side);
    switch (kind) {
    case AMC_K_R: return (s & own) ? s : ST_F;
    case AMC_K_W: return own;
    case AMC_K_PUSH: return (s & own) ? (s | other) : ST_F;
    case AMC_K_PULL: return (s & other) ? (s | own) : ST_F;
    case AMC_K_NOOP: return s;
    case AMC_K_PW: return s & ~other;
    case AMC_K_EN:
        if (s & own) return s;
        return (s & other) ? (s | own) : ST_F;
    }
    return -1;
}

Map make_map(int kind, int side)
{
    Map m(5);
    for (int s = 0; s < 5; ++s) m[s] = (uint8_t)step(kind, side, s);
    return m;
}

Tables build()
{
    Tables t;
    memset(&t, 0, sizeof(t));
    std::vector<Map> gens;
    std::vector<int> gen_byte;
    for (int kind = 0; kind <= AMC_K_EN; ++kind) {
        if (kind == AMC_K_GT) continue;
        for (int side = 0; side < 2; ++side) {
            gens.push_back(make_map(kind, side));
            gen_byte.push_back(kind | side << 4);
        }
    }
    // breadth-first closure under right multiplication by generators
    std::vector<Map> elems;
    std::map<Map, int> id;
    Map ident(5);
    for (int s = 0; s < 5; ++s) ident[s] = (uint8_t)s;
    elems.push_back(ident);
    id[ident] = 0;
    for (size_t i = 0; i < elems.size(); ++i) {
        for (const Map& g : gens) {
            Map c(5);
            for (int s = 0; s < 5; ++s) c[s] = g[elems[i][s]];
            if (!id.count(c)) {
                id[c] = (int)elems.size();
                elems.push_back(c);
            }
        }
    }
    if (elems.size() > (size_t)MAX_ELEMS) abort();
    t.n_elems = (uint8_t)elems.size();
    t.identity = 0;
    for (size_t a = 0; a < elems.size(); ++a) {
        for (int s = 0; s < 5; ++s) t.app[a * 8 + s] = elems[a][s];
        for (size_t b = 0; b < elems.size(); ++b) {
            Map c(5);
            for (int s = 0; s < 5; ++s) c[s] = elems[b][elems[a][s]];
            t.comp[a * MAX_ELEMS + b] = (uint8_t)id.at(c);
        }
    }
    for (int b = 0; b < 256; ++b) t.elem_of[b] = ELEM_BAD;
    for (size_t g = 0; g < gens.size(); ++g) t.elem_of[gen_byte[g]] = (uint8_t)id.at(gens[g]);
    t.elem_of[AMC_K_GT] = ELEM_GT;
    t.elem_of[AMC_K_GT | 16] = ELEM_GT;
    t.pull_of_side[0] = t.elem_of[AMC_K_PULL];          // CPU side: Pull x
    t.pull_of_side[1] = t.elem_of[AMC_K_PULL | 16];     // GPU side: rem Pull = Push x
    return t;
}

}  // namespace

const Tables& host_tables()
{
    static Tables t = build();
    return t;
}

namespace {
SetTables build_sets()
{
    SetTables t;
    memset(&t, 0, sizeof(t));
    for (int kind = 0; kind <= AMC_K_PW; ++kind)
        for (int side = 0; side < 2; ++side) {
            const int o = kind << 1 | side;
            for (int m = 0; m < 32; ++m) {
                uint32_t img = 0;
                for (int s = 0; s < 5; ++s)
                    if (m & (1 << s)) {
                        const int r = step(kind, side, s);
                        img |= 1u << r;
                        if (s != ST_F && r == ST_F) t.flt[o] |= 1u << m;
                    }
                t.img[o * 32 + m] = (uint8_t)img;
            }
        }
    return t;
}
}  // namespace

const SetTables& host_set_tables()
{
    static SetTables t = build_sets();
    return t;
}

namespace {
thread_local cudaEvent_t t_prof_start = nullptr;
thread_local cudaEvent_t t_prof_stop = nullptr;
}  // namespace

void set_profile_events(cudaEvent_t a, cudaEvent_t b)
{
    t_prof_start = a;
    t_prof_stop = b;
}
void profile_begin(cudaStream_t s)
{
    if (t_prof_start) cudaEventRecord(t_prof_start, s);
}
void profile_end(cudaStream_t s)
{
    if (t_prof_stop) cudaEventRecord(t_prof_stop, s);
}

int* device_error_word()
{
    static std::mutex mu;
    static std::map<int, int*> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int* p = nullptr;
    if (cudaGetSymbolAddress((void**)&p, g_error_word) != cudaSuccess) return nullptr;
    cache[dev] = p;
    return p;
}

}  // namespace amc
