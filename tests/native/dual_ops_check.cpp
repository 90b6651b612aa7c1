// The dual-number operations of the tangent path against central differences of the same
// expressions in double, at a few points: prints "name max_relative_error" per operation.
#include <cmath>
#include <cstdio>

#include "fvlbm_dual.h"

using fvlbm::Dual;

template <class F>
static double check(F f, double x) {
    const double h = 1e-6 * (std::fabs(x) + 1.0);
    const double fd = (double(f(Dual(x + h)).v) - double(f(Dual(x - h)).v)) / (2 * h);
    const Dual y = f(Dual(x, 1.0));
    return std::fabs(y.d - fd) / (std::fabs(fd) + 1e-12);
}

int main() {
    const double xs[] = {0.3, 1.7, -2.2, 4.0};
    struct Case {
        const char *name;
        Dual (*f)(Dual);
        bool positive;
    } cases[] = {
        {"mul_add", [](Dual x) { return x * x * Dual(3.0) + x - Dual(1.0); }, false},
        {"div", [](Dual x) { return Dual(2.0) / (x * x + Dual(1.0)); }, false},
        {"sqrt", [](Dual x) { return fvlbm::sqrt(x); }, true},
        {"tanh", [](Dual x) { return fvlbm::tanh(x * Dual(0.7)); }, false},
        {"fmin_fmax", [](Dual x) { return fvlbm::fmin(x * x, Dual(2.0) * x) + fvlbm::fmax(x, -x); }, false},
        {"neg_sub", [](Dual x) { return -(x - x * x * x); }, false},
    };
    for (const Case &c : cases) {
        double worst = 0;
        for (double x : xs) {
            if (c.positive && x <= 0) continue;
            worst = std::fmax(worst, check(c.f, x));
        }
        printf("%s %.3e\n", c.name, worst);
    }
    // sqrt at exactly 0 carries derivative 0 (documented reading, not a limit)
    printf("sqrt0 %.3e\n", fvlbm::sqrt(Dual(0.0, 1.0)).d);
    return 0;
}
