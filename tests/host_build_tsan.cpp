// Driver for the ThreadSanitizer test of the host finite-element build
// (tests/test_host_tsan.py): builds hierarchies with the thread options of
// the device setup (coarsest level on a thread of its own, per-level
// callbacks from two threads) and with those of host-only handles, and
// prints a digest of each so that the test can also compare thread counts.
#include "../paper_2407_07253_gb300/csrc/fem.hpp"

#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <vector>

using namespace sfem;

static Mesh unit_square(int n) {
    Mesh m;
    m.d = 2;
    for (int j = 0; j <= n; ++j)
        for (int i = 0; i <= n; ++i) {
            m.X.push_back(double(i) / n);
            m.X.push_back(double(j) / n);
        }
    m.nv = (n + 1) * (n + 1);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            const int a = j * (n + 1) + i, b = a + 1, c = a + n + 1, d = c + 1;
            m.C.insert(m.C.end(), {a, b, d, a, d, c});
        }
    m.nc = 2 * n * n;
    return m;
}

// the unit cube split into the six Kuhn simplices along its main diagonal
static Mesh kuhn_cube() {
    Mesh m;
    m.d = 3;
    for (int v = 0; v < 8; ++v) {
        m.X.push_back(v & 1);
        m.X.push_back((v >> 1) & 1);
        m.X.push_back((v >> 2) & 1);
    }
    m.nv = 8;
    const int order[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (const auto& p : order) {
        int v = 0;
        m.C.push_back(v);
        for (int q = 0; q < 3; ++q) {
            v |= 1 << p[q];
            m.C.push_back(v);
        }
    }
    m.nc = 6;
    return m;
}

struct Digest {
    unsigned long long h = 1469598103934665603ull;   // FNV-1a
    template <class V>
    void add(const V& v) {
        const unsigned char* c = (const unsigned char*)v.data();
        for (size_t i = 0; i < v.size() * sizeof(v[0]); ++i) {
            h ^= c[i];
            h *= 1099511628211ull;
        }
    }
};

int main() {
    for (int device_like = 0; device_like < 2; ++device_like)
        for (int cfg = 0; cfg < 3; ++cfg) {
            const Mesh coarse = cfg == 2 ? kuhn_cube() : unit_square(4);
            HierarchySpec s;
            s.family = cfg == 1 ? 1 : 0;          // SV on the Alfeld split, else TH
            s.k = cfg == 2 ? 3 : 4;
            s.schedule = {s.k, 2};
            s.n_refine = cfg == 2 ? 2 : 3;
            s.barycentric = cfg == 1;
            s.device_assembly = device_like;
            s.device_transfers = device_like;
            s.coarsest_first = device_like;
            s.coarsest_thread = device_like;
            std::vector<double> nu(1 << 20, 1.0);
            Hierarchy H;
            std::mutex mu;
            long long seen = 0;
            build_hierarchy(coarse, s, nu.data(), H, [&](int l, int stage) {
                std::lock_guard<std::mutex> g(mu);
                const Level& L = H.levels[l];
                seen += stage == 0 ? (long long)L.V.X.size() : (long long)L.patch_dofs.size();
            });
            Digest d;
            for (const Level& L : H.levels) {
                d.add(L.K.rp); d.add(L.K.ci); d.add(L.K.v);
                d.add(L.P.ci); d.add(L.P.v); d.add(L.R.ci); d.add(L.R.v);
                d.add(L.patch_off); d.add(L.patch_dofs);
                d.add(L.V.X); d.add(L.V.cell_nodes); d.add(L.Q.cell_nodes);
                d.add(L.voff); d.add(L.vadj); d.add(L.pint);
            }
            std::printf("%d %d %zu %lld %016llx\n", device_like, cfg, H.levels.size(), seen, d.h);
        }
    return 0;
}
