// Prints the fixed-point shift the library chooses for (entries, max b) pairs
// read from stdin, one "entries max_b" pair per line (host logic only).
#include <cstdio>

#include "../../paper_2002_00352_gb300/csrc/kp_internal.h"

int main() {
    double count;
    float maxb;
    while (std::scanf("%lf %f", &count, &maxb) == 2) std::printf("%d\n", kp::mass_shift(count, maxb));
    return 0;
}
