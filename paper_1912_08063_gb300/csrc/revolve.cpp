// Binomial checkpointing for the reverse sweep (Griewank & Walther, "Algorithm 799:
// revolve", ACM TOMS 26(1), 2000).  The paper names the gradient of the misfit
// (Sec. 1) but not how the forward states reach the reverse sweep; storing all nt
// states does not fit for large grids, so states are checkpointed and recomputed.
//
// Units j = 0..nsteps: the reverse step of unit j needs the forward state S_j (the state
// after j forward steps); units run from nsteps down to 1 (unit 0 needs nothing).  The
// zero initial state S_0 costs no storage.  With c free checkpoint slots, a range
// [a, b) whose first state is available is split at a + l1: advance l1 steps, store,
// reverse [a + l1, b) with c - 1 slots, restore S_a, reverse [a, a + l1) with c slots.
// The minimal number of forward steps for l units and c slots is
//   T(l, c) = r l - beta(c + 2, r - 1),  beta(s, t) = binom(s + t, s),
// with r the least integer such that beta(c + 1, r) >= l; each split is chosen among
// those that reach T exactly.
#include <cstdint>
#include <unordered_map>
#include <vector>

namespace fwi {

namespace {

// binom(s + t, s), saturated at 2^62
int64_t beta(int64_t s, int64_t t)
{
    if (s < 0 || t < 0) return 0;
    const int64_t cap = (int64_t)1 << 62;
    int64_t k = s < t ? s : t, n = s + t;
    __int128 acc = 1;
    for (int64_t i = 1; i <= k; ++i) {
        acc = acc * (n - k + i) / i;
        if (acc > cap) return cap;
    }
    return (int64_t)acc;
}

int64_t min_steps(int64_t l, int64_t c)
{
    if (l <= 1) return 0;
    if (c <= 0) return l * (l - 1) / 2;
    int64_t r = 1;
    while (beta(c + 1, r) < l) ++r;
    return r * l - beta(c + 2, r - 1);
}

struct Builder {
    std::vector<int32_t> out;
    int64_t fwd = 0;
    int64_t maxl = 0;
    std::unordered_map<int64_t, int64_t> memo;  // T(l, c), keyed c * (maxl + 1) + l

    int64_t T(int64_t l, int64_t c)
    {
        if (l <= 1) return 0;
        if (c <= 0) return l * (l - 1) / 2;
        if (c >= l - 1) return l - 1;
        const int64_t key = c * (maxl + 1) + l;
        auto it = memo.find(key);
        if (it != memo.end()) return it->second;
        const int64_t v = min_steps(l, c);
        memo.emplace(key, v);
        return v;
    }
    void emit(int32_t kind, int32_t arg)
    {
        out.push_back(kind);
        out.push_back(arg);
    }
    void advance(int64_t k)
    {
        if (k > 0) {
            emit(1, (int32_t)k);
            fwd += k;
        }
    }

    // Precondition: the current state is S_a; slot_a holds S_a (-1: zero state).
    void rev(int64_t a, int64_t b, int64_t c, int32_t slot_a, int32_t next_free)
    {
        const int64_t l = b - a;
        if (l <= 0) return;
        if (l == 1) {
            if (a > 0) emit(4, (int32_t)a);
            return;
        }
        if (c <= 0) {
            const int64_t jlo = a > 1 ? a : 1;   // unit 0 needs no reverse step
            for (int64_t j = b - 1; j >= jlo; --j) {
                if (j < b - 1) emit(3, slot_a);
                advance(j - a);
                emit(4, (int32_t)j);
            }
            return;
        }
        const int64_t best = T(l, c);
        int64_t l1 = 1;
        for (int64_t t = 1; t < l; ++t) {
            if (t + T(l - t, c - 1) + T(t, c) == best) {
                l1 = t;
                break;
            }
        }
        advance(l1);
        emit(2, next_free);
        rev(a + l1, b, c - 1, next_free, next_free + 1);
        if (a > 0 || l1 > 1) {   // [a, a + l1) holds a unit that needs a reverse step
            emit(3, slot_a);
            rev(a, a + l1, c, slot_a, next_free);
        }
    }
};

}  // namespace

int64_t revolve_min_steps(int64_t units, int64_t slots) { return min_steps(units, slots); }

// Action list for nsteps forward steps (units 0..nsteps) and nslots slots.
std::vector<int32_t> revolve_actions(int32_t nsteps, int32_t nslots, int64_t *n_forward)
{
    Builder b;
    const int64_t units = (int64_t)nsteps + 1;
    int64_t c = nslots < 0 ? 0 : nslots;
    if (c > units) c = units;   // more slots than units never help
    b.maxl = units;
    b.rev(0, units, c, -1, 0);
    if (n_forward) *n_forward = b.fwd;
    return b.out;
}

}  // namespace fwi
