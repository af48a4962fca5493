// Checks of the saved serving-state format (host code only): a round trip, and the errors for
// a corrupted byte, a truncated file, trailing bytes, a wrong magic and a missing file.
// Built and run by tests/test_state_host.py; prints one line per failed check and exits 1 if any.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>

#include "state_io.h"

namespace st = rkm::state;

static int failures = 0;
#define CHECK(cond)                                                          \
    do {                                                                     \
        if (!(cond)) {                                                       \
            std::printf("FAILED %s:%d: %s\n", __FILE__, __LINE__, #cond);    \
            ++failures;                                                      \
        }                                                                    \
    } while (0)

static std::vector<unsigned char> slurp(const std::string& p) {
    std::vector<unsigned char> b;
    FILE* f = std::fopen(p.c_str(), "rb");
    if (!f) return b;
    int c;
    while ((c = std::fgetc(f)) != EOF) b.push_back((unsigned char)c);
    std::fclose(f);
    return b;
}

static void spill(const std::string& p, const std::vector<unsigned char>& b) {
    FILE* f = std::fopen(p.c_str(), "wb");
    if (!b.empty()) std::fwrite(b.data(), 1, b.size(), f);
    std::fclose(f);
}

int main(int argc, char** argv) {
    const std::string dir = argc > 1 ? argv[1] : ".";
    const std::string path = dir + "/state.bin";
    std::mt19937_64 rng(7);
    const int64_t n = 1000;
    const int d = 37;
    std::vector<float> U((size_t)n * d);
    std::vector<double> tau(n);
    std::vector<int32_t> tid(n);
    for (auto& x : U) x = (float)((int)(rng() % 8193) - 4096) / 4096.f;
    for (auto& x : tau) x = (double)(int64_t)(rng() % 100000) / 65536.0 - 0.5;
    for (auto& x : tid) x = (int32_t)(rng() % 50000);
    tau[3] = -0.0;
    std::string err;
    CHECK(st::write(path.c_str(), n, d, U.data(), tau.data(), tid.data(), &err));
    const std::vector<unsigned char> good = slurp(path);
    CHECK(good.size() == 32 + (size_t)n * d * 4 + (size_t)n * 8 + (size_t)n * 4);

    int64_t n2 = 0;
    int d2 = 0;
    std::vector<float> U2;
    std::vector<double> tau2;
    std::vector<int32_t> tid2;
    CHECK(st::read(path.c_str(), &n2, &d2, &U2, &tau2, &tid2, &err));
    CHECK(n2 == n && d2 == d && U2 == U && tid2 == tid);
    CHECK(std::memcmp(tau2.data(), tau.data(), tau.size() * sizeof(double)) == 0);  // bit for bit, -0.0 too

    std::vector<unsigned char> bad = good;
    bad[32 + 1234] ^= 0x10u;  // one payload bit
    spill(path, bad);
    CHECK(!st::read(path.c_str(), &n2, &d2, &U2, &tau2, &tid2, &err) && err.find("hash") != std::string::npos);

    bad = good;
    bad.resize(good.size() - 5);
    spill(path, bad);
    CHECK(!st::read(path.c_str(), &n2, &d2, &U2, &tau2, &tid2, &err) && err.find("truncated") != std::string::npos);

    bad = good;
    bad.push_back(0);
    spill(path, bad);
    CHECK(!st::read(path.c_str(), &n2, &d2, &U2, &tau2, &tid2, &err) && err.find("trailing") != std::string::npos);

    bad = good;
    bad[0] = 'X';
    spill(path, bad);
    CHECK(!st::read(path.c_str(), &n2, &d2, &U2, &tau2, &tid2, &err) && err.find("not a state") != std::string::npos);

    bad = good;
    bad[8] = 2;  // version
    spill(path, bad);
    CHECK(!st::read(path.c_str(), &n2, &d2, &U2, &tau2, &tid2, &err) && err.find("version") != std::string::npos);

    CHECK(!st::read((dir + "/missing.bin").c_str(), &n2, &d2, &U2, &tau2, &tid2, &err));

    // empty resident set
    CHECK(st::write(path.c_str(), 0, 5, nullptr, nullptr, nullptr, &err));
    CHECK(st::read(path.c_str(), &n2, &d2, &U2, &tau2, &tid2, &err) && n2 == 0 && d2 == 5);
    CHECK(!st::write(path.c_str(), 4, 0, U.data(), tau.data(), tid.data(), &err));

    if (failures) return 1;
    std::printf("ok\n");
    return 0;
}
