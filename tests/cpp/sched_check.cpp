// Host check of the Jacobi pair schedules (jacobi_schedule.h): for every
// sweep, each round lists every index exactly once (as a pair member or a
// single), no round has more than m/2 pairs, and every pair (i < j) is
// rotated exactly once per sweep.  Prints "ok <cases>" or the first failure.
#include <algorithm>
#include <cstdio>
#include <set>
#include <utility>
#include <vector>

#include "jacobi_schedule.h"

int main() {
    int cases = 0;
    std::vector<int> sizes;
    for (int n = 1; n <= 40; ++n) sizes.push_back(n);
    for (int n : {47, 48, 64, 99, 184, 185, 300}) sizes.push_back(n);
    for (int n : sizes) {
        mpspt::Sched sc;
        sc.init(n);
        std::set<std::pair<int, int>> pairs;
        if (sc.rounds() > 2 * n + 4) { printf("too many rounds n=%d\n", n); return 1; }
        for (int r = 0; r < sc.rounds(); ++r) {
            const int ns = sc.slots(r);
            if (ns > std::max(n, 1)) { printf("slots %d > n=%d\n", ns, n); return 1; }
            std::vector<int> seen;
            int np = 0;
            for (int k = 0; k < ns; ++k) {
                int p, q;
                sc.slot(r, k, p, q);
                seen.push_back(p);
                if (q >= 0) {
                    if (!(p < q)) { printf("order n=%d\n", n); return 1; }
                    seen.push_back(q);
                    ++np;
                    if (!pairs.insert({p, q}).second) {
                        printf("pair twice n=%d (%d,%d)\n", n, p, q);
                        return 1;
                    }
                }
            }
            std::sort(seen.begin(), seen.end());
            for (int i = 0; i < n; ++i)
                if ((int)seen.size() != n || seen[i] != i) {
                    printf("round misses an index n=%d r=%d\n", n, r);
                    return 1;
                }
            if (np > sc.half) { printf("pairs %d > half n=%d\n", np, n); return 1; }
        }
        if ((long long)pairs.size() != (long long)n * (n - 1) / 2) {
            printf("sweep misses pairs n=%d: %zu\n", n, pairs.size());
            return 1;
        }
        ++cases;
    }
    printf("ok %d\n", cases);
    return 0;
}
