/*
 * op_count.cpp -- operation-counting build of the CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY, like echo_oracle.c itself: it measures how many
 * floating-point operations the method performs per unit of each step (per
 * cell of the inversion, per face of the reconstruction and fluxes, per edge
 * of the EMFs, per cell of the update), so that a kernel's achieved rate can
 * be stated in the method's own operations rather than in the instructions
 * the kernel happens to execute.
 *
 * How: echo_oracle.c is compiled here as C++ with `double` replaced by a
 * number type whose arithmetic operators increment counters.  Counted, each
 * as one operation: +, -, *, / and sqrt.  Not counted: an addition or
 * subtraction with an exact zero operand, a multiplication with an operand
 * of exactly 0 or +-1, a division by +-1 (these are what a flat-space or
 * axis-aligned specialisation omits; in flat space the metric is the
 * identity), negation and |x|, comparisons, min/max and everything inside
 * the scopes the oracle marks OPC_UNCOUNTED (the closed-form metric and its
 * derivatives, grid coordinates, minmod selections).  exp, log, pow, sin
 * and cos are counted apart (they only occur in uncounted scopes or the
 * floors).  The counts are attributed to the step named by the oracle's
 * OPC_PHASE hooks; OPC_UNIT counts the units.  Optionally (cse) an
 * operation is counted once per unit for each distinct kind and pair of
 * operand values, which removes the oracle's recomputation of shared
 * subexpressions (v^2, B^2 and v.B of one state evaluated by the flux, the
 * conserved vector and the speeds alike); and (sample_every) only every
 * k-th unit is counted, the per-unit figure being the counts over the
 * sampled units.  The oracle's loops run under OpenMP as in its plain
 * build; every thread keeps its own counters (a unit runs on one thread),
 * summed when read.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

#include <unordered_set>

namespace opc {
enum { ADD, MUL, DIV, SQRT, FN, NOP };
constexpr int NPH = 9;
constexpr int MAXT = 256;   // OpenMP threads

struct Key {
    int op;
    uint64_t a, b;
    bool operator==(const Key &o) const { return op == o.op && a == o.a && b == o.b; }
};
struct KeyHash {
    size_t operator()(const Key &k) const
    {
        const uint64_t r = (k.a << 31) | (k.a >> 33);
        const uint64_t h = (k.a * 0x9e3779b97f4a7c15ULL) ^ (k.b + 0x632be59bd9b4e019ULL + r);
        return (size_t)(h ^ ((uint64_t)k.op * 0xbf58476d1ce4e5b9ULL));
    }
};

// Counters of one OpenMP thread (the oracle's loops run in parallel; each
// unit is handled by one thread from start to end).
struct alignas(64) Slot {
    long long count[NPH][NOP];
    long long units[NPH];      // units of each step
    long long sampled[NPH];    // of those, the units whose operations were counted
    int paused;                // depth of open uncounted scopes
    bool in_unit;              // a unit of the current step is open
    bool in_sample;
    std::unordered_set<Key, KeyHash> seen;   // operations of the open unit
};
Slot slot[MAXT];
int phase = NPH - 1;        // set outside parallel regions, read inside
int sample_every = 1;       // count the operations of every k-th unit only
bool cse = false;           // count each distinct (operation, operands) once per unit

inline Slot &me() { return slot[omp_get_thread_num()]; }

inline uint64_t bits(double x)
{
    uint64_t u;
    memcpy(&u, &x, sizeof u);
    return u;
}

__attribute__((noinline)) void add_slow(Slot &t, int op, int key, double a, double b)
{
    if (cse && t.in_unit) {
        if (!t.seen.insert(Key{key, bits(a), bits(b)}).second)
            return;
    }
    ++t.count[phase][op];
}

// One operation of kind `op` (key: the distinguishing code, e.g. ADD and SUB
// apart) on operands a, b (b = 0 for a unary one).
inline void add(int op, int key, double a, double b)
{
    Slot &t = me();
    if (t.paused || !t.in_sample)
        return;
    add_slow(t, op, key, a, b);
}

inline void set_phase(int k)
{
    phase = k;
    for (int i = 0; i < MAXT; ++i) {
        slot[i].in_unit = false;
        slot[i].in_sample = true;
        if (!slot[i].seen.empty())
            slot[i].seen.clear();
    }
}

inline void unit()
{
    Slot &t = me();
    if (t.paused)
        return;
    const long long u = t.units[phase]++;
    t.in_unit = true;
    t.in_sample = (u % sample_every) == 0;
    if (t.in_sample)
        ++t.sampled[phase];
    if (!t.seen.empty())
        t.seen.clear();
}

struct Uncounted {
    Uncounted() { ++me().paused; }
    ~Uncounted() { --me().paused; }
};
}  // namespace opc

struct cdbl {
    double v;
    cdbl() = default;
    cdbl(double x) : v(x) {}
    explicit operator double() const { return v; }
    cdbl &operator+=(cdbl b);
    cdbl &operator-=(cdbl b);
    cdbl &operator*=(cdbl b);
    cdbl &operator/=(cdbl b);
};

inline bool unit_or_zero(double a) { return a == 0.0 || a == 1.0 || a == -1.0; }

enum { K_ADD, K_SUB, K_MUL, K_DIV, K_SQRT };

inline cdbl operator+(cdbl a, cdbl b)
{
    if (a.v != 0.0 && b.v != 0.0)
        opc::add(opc::ADD, K_ADD, a.v < b.v ? a.v : b.v, a.v < b.v ? b.v : a.v);
    return cdbl(a.v + b.v);
}
inline cdbl operator-(cdbl a, cdbl b)
{
    if (a.v != 0.0 && b.v != 0.0)
        opc::add(opc::ADD, K_SUB, a.v, b.v);
    return cdbl(a.v - b.v);
}
inline cdbl operator*(cdbl a, cdbl b)
{
    if (!unit_or_zero(a.v) && !unit_or_zero(b.v))
        opc::add(opc::MUL, K_MUL, a.v < b.v ? a.v : b.v, a.v < b.v ? b.v : a.v);
    return cdbl(a.v * b.v);
}
inline cdbl operator/(cdbl a, cdbl b)
{
    if (b.v != 1.0 && b.v != -1.0 && a.v != 0.0)
        opc::add(opc::DIV, K_DIV, a.v, b.v);
    return cdbl(a.v / b.v);
}
inline cdbl operator-(cdbl a) { return cdbl(-a.v); }
inline cdbl operator+(cdbl a) { return a; }
inline cdbl &cdbl::operator+=(cdbl b) { return *this = *this + b; }
inline cdbl &cdbl::operator-=(cdbl b) { return *this = *this - b; }
inline cdbl &cdbl::operator*=(cdbl b) { return *this = *this * b; }
inline cdbl &cdbl::operator/=(cdbl b) { return *this = *this / b; }
inline bool operator<(cdbl a, cdbl b) { return a.v < b.v; }
inline bool operator>(cdbl a, cdbl b) { return a.v > b.v; }
inline bool operator<=(cdbl a, cdbl b) { return a.v <= b.v; }
inline bool operator>=(cdbl a, cdbl b) { return a.v >= b.v; }
inline bool operator==(cdbl a, cdbl b) { return a.v == b.v; }
inline bool operator!=(cdbl a, cdbl b) { return a.v != b.v; }

inline cdbl sqrt(cdbl a)
{
    opc::add(opc::SQRT, K_SQRT, a.v, 0.0);
    return cdbl(::sqrt(a.v));
}
inline cdbl fabs(cdbl a) { return cdbl(::fabs(a.v)); }
inline cdbl fmin(cdbl a, cdbl b) { return cdbl(::fmin(a.v, b.v)); }
inline cdbl fmax(cdbl a, cdbl b) { return cdbl(::fmax(a.v, b.v)); }
inline cdbl exp(cdbl a)
{
    opc::add(opc::FN, 100, a.v, 0.0);
    return cdbl(::exp(a.v));
}
inline cdbl log(cdbl a)
{
    opc::add(opc::FN, 101, a.v, 0.0);
    return cdbl(::log(a.v));
}
inline cdbl pow(cdbl a, cdbl b)
{
    opc::add(opc::FN, 102, a.v, b.v);
    return cdbl(::pow(a.v, b.v));
}
inline cdbl sin(cdbl a)
{
    opc::add(opc::FN, 103, a.v, 0.0);
    return cdbl(::sin(a.v));
}
inline cdbl cos(cdbl a)
{
    opc::add(opc::FN, 104, a.v, 0.0);
    return cdbl(::cos(a.v));
}

#define OPC_PHASE(k) opc::set_phase(k)
#define OPC_UNIT() opc::unit()
#define OPC_UNCOUNTED opc::Uncounted opc_uncounted_scope_
#define double cdbl

extern "C" {
#include "echo_oracle.c"

/* Zero the counters.  sample_every: count the operations of every k-th
 * unit of each step only (k >= 1); cse: count each distinct operation
 * (kind and operand values) once per unit -- the operations left when
 * every repeated subexpression of the oracle's formulas is computed once. */
void oracle_count_reset(int sample_every, int cse)
{
    for (int i = 0; i < opc::MAXT; ++i) {
        opc::Slot &t = opc::slot[i];
        memset(t.count, 0, sizeof(t.count));
        memset(t.units, 0, sizeof(t.units));
        memset(t.sampled, 0, sizeof(t.sampled));
        t.paused = 0;
        std::unordered_set<opc::Key, opc::KeyHash>().swap(t.seen);   // drop a grown bucket array
    }
    opc::sample_every = sample_every > 0 ? sample_every : 1;
    opc::cse = cse != 0;
    opc::set_phase(OPC_OTHER);
}

/* counts: OPC_NPHASE x 5 (add, mul, div, sqrt, other functions) since the
 * last reset, summed over threads; units and sampled: OPC_NPHASE each. */
void oracle_count_read(long long *counts, long long *units, long long *sampled)
{
    for (int p = 0; p < OPC_NPHASE; ++p) {
        for (int o = 0; o < opc::NOP; ++o)
            counts[p * opc::NOP + o] = 0;
        units[p] = sampled[p] = 0;
        for (int i = 0; i < opc::MAXT; ++i) {
            for (int o = 0; o < opc::NOP; ++o)
                counts[p * opc::NOP + o] += opc::slot[i].count[p][o];
            units[p] += opc::slot[i].units[p];
            sampled[p] += opc::slot[i].sampled[p];
        }
    }
}

int oracle_count_nphase(void) { return OPC_NPHASE; }
}
