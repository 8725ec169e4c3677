// rmat_internal.h -- internal types shared by the librmat translation units.
#pragma once

#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "rmat.h"

namespace rmat {

// One alias table: the canonical list of paths plus its alias structure
// (one per level group for per-level tables).
struct PathTable {
    int n0 = 2;                    // initiator size: symbols are the n0^2 cells
    int entries = 0;               // |Q|
    int bits = 0;                  // b, padded size N = 2^b
    int max_len = 0;               // longest path (levels)
    int min_len = 0;               // shortest path with non-zero weight
    std::vector<uint64_t> sym;     // path symbols, top level in bits 63..62 (n0 = 2);
                                   // n0 > 2: base-n0^2 digits, left-aligned in
                                   // kron_depth_cap(n0) digits (kron_symbol)
    std::vector<uint8_t> len;      // path length (levels)
    std::vector<double> p;         // FP64 path probability
    std::vector<uint64_t> w;       // u32 weight, sum 2^32
    std::vector<uint32_t> thr;     // alias threshold, < 2^(32-b)
    std::vector<uint32_t> alias;   // alias target
};

constexpr int kMaxGroups = 64;                 // level groups per table
constexpr size_t kHeaderWords = 4 * kMaxGroups; // blob header: A, B-self, B-alias offsets, bits

// Device table image formats (see rmat_image.cpp).
enum ImageFormat : int {
    kCompact = 0,  // paths <= 13 levels: A = (thr << b) | alias (u32), B = packed path (u32)
    kWide = 1,     // paths <= 32 levels: A as above, B = {row bits, col bits, len, 0} (uint4)
    kKron = 2      // n0 > 2: AA = {A, alias} (uint2), P = {row digits, col digits, len, n0^len - 1} (uint4)
};

struct GroupDesc {
    uint32_t a_off_words;   // offset of A in the image, in u32 words
    uint32_t bs_off_words;  // offset of B-self (path of column j)
    uint32_t ba_off_words;  // offset of B-alias (path of alias[j])
    int bits;
    int len;               // levels of this group (per-level tables)
};

struct DeviceCopy {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// Launch shape of the sampling kernel for one table on one device.
struct AliasPlan {
    int fmt = 0;
    bool u64 = false;
    bool levels = false;
    bool smem_table = true;
    int threads = 0;
    int tile = 0;
    int ctas_per_sm = 0;
    int sms = 0;
    size_t smem_bytes = 0;
    void *kernel = nullptr;
    void *fast_kernel = nullptr;  // the contract-case kernel, when the table qualifies
    size_t fast_smem_bytes = 0;   // its shared memory, when it differs from smem_bytes (Kronecker)
    unsigned *err = nullptr;
};

}  // namespace rmat

struct rmat_table {
    int k = 0;
    int n0 = 2;                             // initiator size (2 = R-MAT)
    unsigned flags = 0;
    bool per_level = false;                 // draw g uses group g
    std::vector<rmat::PathTable> groups;
    int format = rmat::kCompact;
    std::vector<uint32_t> image;            // host copy of the device image
    std::vector<rmat::GroupDesc> gdesc;
    std::mutex mu;
    std::map<int, rmat::DeviceCopy> dev;    // device ordinal -> copy
    bool has_params = false;                // one (a, b, c, d) for every level
    double params[4] = {0, 0, 0, 0};        // ... normalised (partition splits)
    bool scramble = false;                  // relabel vertex IDs
    uint64_t scr[6] = {0, 0, 0, 0, 0, 0};   // m0, a0, m1, a1, m2, a2
    bool cfg_set = false;
    rmat_launch_config_t cfg{};
    std::map<int, rmat::AliasPlan> plans;   // device ordinal -> launch plan
};

namespace rmat {

// Thread-local error message; returns `st` for convenient `return fail(...)`.
rmat_status fail(rmat_status st, const std::string &msg);
void clear_error();

// Table construction (rmat_table.cpp).
rmat_status build_variable(const double P[4], int k, uint64_t bound, PathTable &out);
// Stochastic Kronecker tables with an n0 x n0 initiator P (row-major, normalised).
rmat_status build_kron_variable(const double *P, int n0, int k, uint64_t bound, PathTable &out);
rmat_status build_kron_fixed(const double *P, int n0, int ell, PathTable &out);
rmat_status normalise_theta(const double *in, int n0, std::vector<double> &out);
int kron_depth_cap(int n0);   // largest L with n0^L <= 2^32
int kron_max_k(int n0);       // largest k with n0^k <= 2^64
// Symbol of `level` in the left-aligned base-n0^2 key of a Kronecker path.
uint32_t kron_symbol(uint64_t key, int n0, int level);
// Whether the table's vertex IDs need 64 bits (n0^k > 2^32).
bool wide_ids(const rmat_table *t);
// Bits per coordinate of the packed Kronecker path (u32 IDs, digits of the
// longest path in S bits, 2S + 4 <= 32, paths of at most 15 levels); 0 when the
// table does not pack.
int kron_packed_shift(const rmat_table *t);
rmat_status build_fixed(const double *P_levels, int ell, PathTable &out);
rmat_status normalise_params(const double in[4], double out[4]);

// Device image (rmat_image.cpp): fills t->image / t->gdesc / t->format.
rmat_status build_image(rmat_table *t);

// Upload of the image for the current device (rmat_api.cu).
rmat_status ensure_device_copy(const rmat_table *t, const uint32_t **dptr);
// The table's launch plan on the current device (cached) and its device image.
rmat_status plan_and_image(const rmat_table *t, AliasPlan &plan, const uint32_t **img);

}  // namespace rmat
