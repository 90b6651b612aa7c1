// Host-side check of the adjoint's checkpoint schedule (revolve_schedule): for a range of unit
// and snapshot counts, simulate the actions on snapshot contents and check that every unit is
// reversed exactly once, last to first, from a snapshot that holds its start state; that no
// snapshot index reaches the count; and that the forward work stays within the binomial bound
// (r + 1) units, r the least number with C(snaps + r, snaps) >= units.  Prints one line per
// case, "ok" or the failure, then the total forward passes of a few cases.
#include <cstdio>
#include <vector>

#include "fvlbm_internal.h"

using namespace fvlbm;

static double binom(int c, int r) {
    double b = 1.0;
    for (int i = 1; i <= c; ++i) b = b * (r + i) / i;
    return b;
}

static const char *check(int units, int snaps, long *passes) {
    std::vector<RevolveAction> plan;
    const bool ok = revolve_schedule(units, snaps, &plan);
    if (units >= 2 && snaps == 0) return ok ? "schedule without snapshots" : "ok";
    if (!ok) return "refused";
    std::vector<int> holds(snaps, -1);  // unit whose start state each snapshot holds
    int next = units - 1;
    long work = 0;
    for (const RevolveAction &a : plan) {
        const int at = a.from < 0 ? 0 : (a.from < snaps ? holds[a.from] : -2);
        if (at != a.u0) return "action from a snapshot that does not hold its start";
        if (a.kind == RevolveAction::kAdvance) {
            if (a.to < 0 || a.to >= snaps || a.u1 <= a.u0 || a.u1 > units) return "bad advance";
            holds[a.to] = a.u1;
            work += a.u1 - a.u0;
        } else {
            if (a.u0 != next) return "units not reversed last to first";
            --next;
            work += 1;
        }
    }
    if (next != -1) return "not every unit reversed";
    int r = 0;
    while (binom(snaps, r) < units) ++r;
    if (work > static_cast<long>(r + 1) * units) return "forward work above the binomial bound";
    *passes = work;
    return "ok";
}

int main() {
    int bad = 0;
    for (int units = 0; units <= 60; ++units)
        for (int snaps = 0; snaps <= 8; ++snaps) {
            long p = 0;
            const char *r = check(units, snaps, &p);
            if (r[0] != 'o' || r[1] != 'k') {
                printf("units %d snaps %d: %s\n", units, snaps, r);
                ++bad;
            }
        }
    const int big[][2] = {{1000, 5}, {1000, 30}, {5000, 10}, {100, 3}, {17, 16}};
    for (const auto &c : big) {
        long p = 0;
        const char *r = check(c[0], c[1], &p);
        if (r[0] != 'o' || r[1] != 'k') {
            printf("units %d snaps %d: %s\n", c[0], c[1], r);
            ++bad;
        }
        printf("passes %d %d %ld\n", c[0], c[1], p);
    }
    printf(bad ? "FAILED\n" : "ok\n");
    return bad ? 1 : 0;
}
