// Stress driver for the library's host worker pool (csrc/host_pool.h), built by
// tests/test_host_pool.py with the host compiler. Checks that every job of a
// call runs exactly once and that the call returns only after all of them,
// for one caller and for several host threads calling at once.
#include <atomic>
#include <cstdio>
#include <thread>
#include <vector>

#include "host_pool.h"

int main() {
    pb::HostPool pool(7);
    long bad = 0;
    for (int it = 0; it < 20000; ++it) {
        const int n = 1 + it % 19;
        std::vector<int> hit(n, 0);
        pool.run(n, [&](int i) { hit[i]++; });
        for (int i = 0; i < n; ++i) bad += hit[i] != 1;
    }
    std::atomic<long> cbad{0};
    std::vector<std::thread> callers;
    for (int c = 0; c < 4; ++c)
        callers.emplace_back([&, c] {
            for (int it = 0; it < 5000; ++it) {
                const int n = 1 + (it + c) % 13;
                std::vector<std::atomic<int>> hit(n);
                for (auto& h : hit) h = 0;
                pool.run(n, [&](int i) { hit[i]++; });
                for (int i = 0; i < n; ++i) cbad += hit[i] != 1;
            }
        });
    for (auto& t : callers) t.join();
    std::printf("single caller %ld bad, concurrent callers %ld bad\n", bad, cbad.load());
    return (bad || cbad.load()) ? 1 : 0;
}
