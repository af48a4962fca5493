// File format of a saved serving state (host code only; no CUDA).
//
// The serving state of a context is its resident users and their thresholds: U (n x d FP32),
// tau_u (FP64) and t_u (int32) as given to rkm_resident_set.  Everything else the serving
// loop keeps on the device (norms, grid codes, ratio order, operand packs) is derived from
// them in milliseconds, so a saved state holds only these three arrays; loading one replays
// rkm_resident_set and skips the threshold pass, which is the expensive part (the paper's
// pre-processing, done once, Section 4).
//
// Layout (little-endian, as on both x86-64 and AArch64):
//   bytes 0..7    magic "RKMSTAT1"
//   bytes 8..11   format version (1)
//   bytes 12..15  d
//   bytes 16..23  n
//   bytes 24..31  FNV-1a 64-bit hash of the payload
//   payload       U[n][d] float32, tau[n] float64, tid[n] int32
#pragma once

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace rkm {
namespace state {

constexpr char MAGIC[8] = {'R', 'K', 'M', 'S', 'T', 'A', 'T', '1'};
constexpr uint32_t VERSION = 1;
constexpr int64_t MAX_N = (int64_t)1 << 31;
constexpr int MAX_D = 256;

// FNV-1a over a byte range, continuing from h.
inline uint64_t fnv1a(const void* data, size_t bytes, uint64_t h = 1469598103934665603ull) {
    const unsigned char* p = static_cast<const unsigned char*>(data);
    for (size_t i = 0; i < bytes; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

inline uint64_t payload_hash(int64_t n, int d, const float* U, const double* tau, const int32_t* tid) {
    uint64_t h = fnv1a(U, (size_t)n * (size_t)d * sizeof(float));
    h = fnv1a(tau, (size_t)n * sizeof(double), h);
    return fnv1a(tid, (size_t)n * sizeof(int32_t), h);
}

struct File {
    FILE* f = nullptr;
    explicit File(FILE* f_) : f(f_) {}
    ~File() {
        if (f) std::fclose(f);
    }
};

// Write a state file; false with a message in *err on failure (the file may then be partial).
inline bool write(const char* path, int64_t n, int d, const float* U, const double* tau, const int32_t* tid,
                  std::string* err) {
    if (n < 0 || n > MAX_N || d < 1 || d > MAX_D) {
        *err = "state: bad shape";
        return false;
    }
    File fh(std::fopen(path, "wb"));
    if (!fh.f) {
        *err = std::string("state: cannot open ") + path + " for writing";
        return false;
    }
    const uint32_t ver = VERSION, dd = (uint32_t)d;
    const uint64_t hash = payload_hash(n, d, U, tau, tid);
    bool ok = std::fwrite(MAGIC, 1, 8, fh.f) == 8 && std::fwrite(&ver, 4, 1, fh.f) == 1 &&
              std::fwrite(&dd, 4, 1, fh.f) == 1 && std::fwrite(&n, 8, 1, fh.f) == 1 &&
              std::fwrite(&hash, 8, 1, fh.f) == 1;
    if (ok && n > 0)
        ok = std::fwrite(U, sizeof(float) * (size_t)d, (size_t)n, fh.f) == (size_t)n &&
             std::fwrite(tau, sizeof(double), (size_t)n, fh.f) == (size_t)n &&
             std::fwrite(tid, sizeof(int32_t), (size_t)n, fh.f) == (size_t)n;
    if (ok) ok = std::fflush(fh.f) == 0;
    if (!ok) *err = std::string("state: write to ") + path + " failed";
    return ok;
}

// Read a state file written by write(); false with a message in *err when the file cannot be
// read, is not a state file of this version, is truncated or fails its hash.
inline bool read(const char* path, int64_t* n, int* d, std::vector<float>* U, std::vector<double>* tau,
                 std::vector<int32_t>* tid, std::string* err) {
    File fh(std::fopen(path, "rb"));
    if (!fh.f) {
        *err = std::string("state: cannot open ") + path;
        return false;
    }
    char magic[8];
    uint32_t ver = 0, dd = 0;
    int64_t nn = 0;
    uint64_t hash = 0;
    if (std::fread(magic, 1, 8, fh.f) != 8 || std::memcmp(magic, MAGIC, 8) != 0) {
        *err = "state: not a state file";
        return false;
    }
    if (std::fread(&ver, 4, 1, fh.f) != 1 || ver != VERSION) {
        *err = "state: unsupported format version";
        return false;
    }
    if (std::fread(&dd, 4, 1, fh.f) != 1 || std::fread(&nn, 8, 1, fh.f) != 1 || std::fread(&hash, 8, 1, fh.f) != 1 ||
        nn < 0 || nn > MAX_N || dd < 1 || dd > (uint32_t)MAX_D) {
        *err = "state: bad header";
        return false;
    }
    U->resize((size_t)nn * dd);
    tau->resize((size_t)nn);
    tid->resize((size_t)nn);
    if (nn > 0 && (std::fread(U->data(), sizeof(float) * dd, (size_t)nn, fh.f) != (size_t)nn ||
                   std::fread(tau->data(), sizeof(double), (size_t)nn, fh.f) != (size_t)nn ||
                   std::fread(tid->data(), sizeof(int32_t), (size_t)nn, fh.f) != (size_t)nn)) {
        *err = "state: truncated file";
        return false;
    }
    char extra;
    if (std::fread(&extra, 1, 1, fh.f) != 0) {
        *err = "state: trailing bytes after the payload";
        return false;
    }
    if (payload_hash(nn, (int)dd, U->data(), tau->data(), tid->data()) != hash) {
        *err = "state: payload hash mismatch (corrupted file)";
        return false;
    }
    *n = nn;
    *d = (int)dd;
    return true;
}

}  // namespace state
}  // namespace rkm
