// Internal helpers shared by the library's translation units: status handling,
// device buffers and the tree / plan structures behind the opaque handles.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "../../include/kifmm.h"

namespace kifmm {

void set_error(const char* fmt, ...);
void clear_error();

struct Status {
    int code = KIFMM_OK;
};

// Throw-free error propagation: each macro records a message and returns a status.
#define KF_CHECK_CUDA(call)                                                        \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            kifmm::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,            \
                             cudaGetErrorString(e_));                              \
            return (e_ == cudaErrorMemoryAllocation) ? KIFMM_ERR_OOM : KIFMM_ERR_CUDA; \
        }                                                                          \
    } while (0)

#define KF_CHECK_LAUNCH()                                                          \
    do {                                                                           \
        cudaError_t e_ = cudaGetLastError();                                       \
        if (e_ != cudaSuccess) {                                                   \
            kifmm::set_error("%s:%d kernel launch: %s", __FILE__, __LINE__,        \
                             cudaGetErrorString(e_));                              \
            return KIFMM_ERR_CUDA;                                                 \
        }                                                                          \
    } while (0)

#define KF_TRY(expr)                                                               \
    do {                                                                           \
        int rc_ = (expr);                                                          \
        if (rc_ != KIFMM_OK) return rc_;                                           \
    } while (0)

#define KF_ARG(cond, msg)                                                          \
    do {                                                                           \
        if (!(cond)) {                                                             \
            kifmm::set_error("invalid argument: %s", msg);                         \
            return KIFMM_ERR_INVALID_ARG;                                          \
        }                                                                          \
    } while (0)

// Owned device allocation (freed in the destructor).
template <typename T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    int alloc(size_t count) {
        release();
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc((void**)&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            set_error("cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
            return KIFMM_ERR_OOM;
        }
        n = count;
        return KIFMM_OK;
    }
    size_t bytes() const { return n * sizeof(T); }
    int upload(const std::vector<T>& h, cudaStream_t s) {
        KF_TRY(alloc(h.size()));
        if (!h.empty())
            KF_CHECK_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T),
                                          cudaMemcpyHostToDevice, s));
        return KIFMM_OK;
    }
};

template <typename T>
int download(std::vector<T>& h, const T* d, size_t n, cudaStream_t s) {
    h.resize(n);
    if (n) {
        KF_CHECK_CUDA(cudaMemcpyAsync(h.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost, s));
        KF_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    return KIFMM_OK;
}

constexpr int kMaxDepth = 20;       // deepest octree level
constexpr int kKeyBits = 21;        // Morton bits per axis
constexpr double kDelta = 1e-5;     // tolerance radius of the singular pair (Sec. III.A.1)
constexpr int kNumOffsets = 343;    // (dx, dy, dz) in [-3, 3]^3 -> (dx+3)*49 + (dy+3)*7 + (dz+3)

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Tree: sorted points, boxes (level-major, Morton-sorted within a level) and
// interaction lists in CSR form (target box -> source boxes).
struct Tree {
    int device = 0;
    int64_t ns = 0, nt = 0;
    bool same = true;                   // targets are the sources
    int max_leaf = 0;
    int forest_level = -1;              // forest: level whose boxes are the instances
    std::vector<int64_t> inst_off;      // forest: instance i owns input points [inst_off[i], inst_off[i+1])
    double root_c[3] = {0, 0, 0};
    double root_h = 0;                  // half-width of the root cube
    int nbox = 0, nlev = 0, nleaf = 0;
    std::vector<int> level_off;         // host: boxes of level l are [level_off[l], level_off[l+1])
    std::vector<double> level_half;     // host: half-width per level

    DBuf<double> sxyz, txyz;            // sorted coordinates, SoA (3*n)
    DBuf<int64_t> sperm, tperm;         // sorted position -> input index
    DBuf<uint64_t> skey, tkey;

    DBuf<int> lvl, coord, parent, child, leaf;  // coord: 3 per box, child: 8 per box
    DBuf<uint64_t> code;                // Morton code at the box's level
    DBuf<int64_t> rng;                  // 4 per box: sbeg, send, tbeg, tend
    DBuf<double> ctr;                   // 3 per box: centre

    DBuf<int> u_off, u_idx, v_off, v_idx, w_off, w_idx, x_off, x_idx;  // CSR (int32)
    int64_t nu = 0, nv = 0, nw = 0, nx = 0, p2p_pairs = 0;

    // Host copies used to build plans.
    std::vector<int> h_lvl, h_parent, h_leaf, h_coord, h_child;
    std::vector<int64_t> h_rng;
    std::vector<int> h_u_off, h_u_idx, h_v_off, h_v_idx, h_w_off, h_w_idx, h_x_off, h_x_idx;
    std::vector<double> h_ctr;
};

}  // namespace kifmm

struct kifmm_tree_s {
    kifmm::Tree t;
};
