// Driver for tests/test_host_reference_tensors.py: prints the library's
// reference element (lattice multi-indices) and reference tensors (M, S, Cq,
// qint of the degree-k velocity / degree k-1 pressure pair) for one (d, k);
// with a third argument, the basis values at the points read from stdin.
#include "../paper_2407_07253_gb300/csrc/fem.hpp"

#include <cstdio>
#include <cstdlib>

int main(int argc, char** argv) {
    if (argc != 3 && argc != 4) return 2;
    const int d = std::atoi(argv[1]), k = std::atoi(argv[2]);
    const sfem::RefElement& v = sfem::reference_element(d, k);
    if (argc == 4) {
        // "eval": read points xi (d numbers each) from stdin, print the basis
        // values at each, in the order of the lattice multi-indices printed first
        for (const auto& a : v.alpha) std::printf("%d %d %d %d\n", a[0], a[1], a[2], a[3]);
        double xi[3] = {0, 0, 0}, out[320];
        for (;;) {
            for (int c = 0; c < d; ++c)
                if (std::scanf("%lf", &xi[c]) != 1) return 0;
            v.eval(xi, out);
            for (int i = 0; i < v.nb; ++i) std::printf("%.17g%c", out[i], i + 1 < v.nb ? ' ' : '\n');
        }
    }
    const sfem::RefElement& q = sfem::reference_element(d, k - 1);
    sfem::RefTensors t;
    t.init(v, q);
    std::printf("%d %d\n", v.nb, q.nb);
    for (const auto& a : v.alpha) std::printf("%d %d %d %d\n", a[0], a[1], a[2], a[3]);
    for (const auto& a : q.alpha) std::printf("%d %d %d %d\n", a[0], a[1], a[2], a[3]);
    for (double x : t.M) std::printf("%.17g\n", x);
    for (double x : t.S) std::printf("%.17g\n", x);
    for (double x : t.Cq) std::printf("%.17g\n", x);
    for (double x : t.qint) std::printf("%.17g\n", x);
    return 0;
}
