// Adaptive octree and interaction lists on the device.
//
// The paper inserts target and source points into one octree whose height sets the
// balance of near- and far-field work (Sec. III.A.1, target-source model; Sec. IV.A,
// the height tuned per problem).  Here the height follows from a leaf capacity:
// points are sorted by Morton key (Sec. III.B: Morton/z-order) and a box is split
// while it holds more than max_leaf sources or targets.  Lists follow the adaptive
// KIFMM of Ying, Biros & Zorin (J. Comput. Phys. 196, 2004):
//   U(B), B leaf:  leaves adjacent to B (B included)
//   V(B):          children of the colleagues of parent(B) not adjacent to B
//   W(B), B leaf:  descendants of B's colleagues not adjacent to B whose parent is
//   X(B):          leaves A with B in W(A), i.e. leaves no finer than parent(B),
//                  adjacent to parent(B) and not adjacent to B
// Only pairs with sources on the source side and targets on the target side are kept.
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace kifmm {

namespace {

__host__ __device__ inline uint64_t spread3(uint64_t v) {
    v &= 0x1fffffULL;
    v = (v | (v << 32)) & 0x1f00000000ffffULL;
    v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
    v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
    v = (v | (v << 2)) & 0x1249249249249249ULL;
    return v;
}

__host__ __device__ inline uint64_t morton3(uint64_t x, uint64_t y, uint64_t z) {
    return (spread3(x) << 2) | (spread3(y) << 1) | spread3(z);
}

struct LevelTable {
    int off[kMaxDepth + 3];
    int nlev;
};

__global__ void k_bbox_partial(const double* __restrict__ xyz, int64_t n, double* part) {
    __shared__ double s[6][256];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int d = 0; d < 3; ++d) {
            double v = xyz[d * n + i];
            if (!isfinite(v)) bad = true;
            lo[d] = fmin(lo[d], v);
            hi[d] = fmax(hi[d], v);
        }
    }
    if (bad) lo[0] = NAN;
    for (int d = 0; d < 3; ++d) {
        s[d][threadIdx.x] = lo[d];
        s[3 + d][threadIdx.x] = hi[d];
    }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            for (int d = 0; d < 3; ++d) {
                double a = s[d][threadIdx.x], b = s[d][threadIdx.x + w];
                s[d][threadIdx.x] = (isnan(a) || isnan(b)) ? NAN : fmin(a, b);
                s[3 + d][threadIdx.x] = fmax(s[3 + d][threadIdx.x], s[3 + d][threadIdx.x + w]);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 6; ++d) part[blockIdx.x * 6 + d] = s[d][0];
}

__global__ void k_morton(const double* __restrict__ xyz, int64_t n, double x0, double y0,
                         double z0, double inv_cell, uint64_t* key, int64_t* idx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double lim = (double)((1u << kKeyBits) - 1);
    double fx = fmin(fmax(floor((xyz[i] - x0) * inv_cell), 0.0), lim);
    double fy = fmin(fmax(floor((xyz[n + i] - y0) * inv_cell), 0.0), lim);
    double fz = fmin(fmax(floor((xyz[2 * n + i] - z0) * inv_cell), 0.0), lim);
    key[i] = morton3((uint64_t)fx, (uint64_t)fy, (uint64_t)fz);
    idx[i] = i;
}

__global__ void k_gather_xyz(const double* __restrict__ in, const int64_t* __restrict__ perm,
                             int64_t n, double* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    out[i] = in[j];
    out[n + i] = in[n + j];
    out[2 * n + i] = in[2 * n + j];
}

__device__ inline int64_t lower_bound_u64(const uint64_t* a, int64_t lo, int64_t hi, uint64_t v) {
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One thread per (box of this level, octant): child ranges and a non-empty flag.
__global__ void k_split_count(int off, int nlevbox, int level, int max_leaf, int force_level, bool same,
                              const uint64_t* __restrict__ skey, const uint64_t* __restrict__ tkey,
                              const uint64_t* __restrict__ code, const int64_t* __restrict__ rng,
                              int* __restrict__ leaf, int* __restrict__ flag,
                              int64_t* __restrict__ crng) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nlevbox * 8) return;
    int b = off + g / 8, oct = g % 8;
    int64_t sb = rng[4 * b], se = rng[4 * b + 1], tb = rng[4 * b + 2], te = rng[4 * b + 3];
    // a forest splits every box above its instance level, whatever it holds
    bool split = (max(se - sb, te - tb) > max_leaf || level < force_level) && (se > sb || te > tb) &&
                 (level < kMaxDepth);
    if (oct == 0) leaf[b] = split ? 0 : 1;
    if (!split) {
        flag[g] = 0;
        return;
    }
    uint64_t cc = code[b] * 8 + oct;
    int shift = 3 * (kKeyBits - (level + 1));
    uint64_t lo = cc << shift, hi = (cc + 1) << shift;
    int64_t csb = lower_bound_u64(skey, sb, se, lo), cse = lower_bound_u64(skey, csb, se, hi);
    int64_t ctb, cte;
    if (same) {
        ctb = csb;
        cte = cse;
    } else {
        ctb = lower_bound_u64(tkey, tb, te, lo);
        cte = lower_bound_u64(tkey, ctb, te, hi);
    }
    crng[4 * g] = csb;
    crng[4 * g + 1] = cse;
    crng[4 * g + 2] = ctb;
    crng[4 * g + 3] = cte;
    flag[g] = (cse > csb || cte > ctb) ? 1 : 0;
}

__global__ void k_split_emit(int off, int nlevbox, int level, int next_off,
                             const int* __restrict__ flag, const int* __restrict__ pos,
                             const int64_t* __restrict__ crng, double x0, double y0, double z0,
                             double child_cell, int* __restrict__ lvl, int* __restrict__ coord,
                             int* __restrict__ parent, int* __restrict__ child,
                             uint64_t* __restrict__ code, int64_t* __restrict__ rng,
                             double* __restrict__ ctr) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nlevbox * 8) return;
    int b = off + g / 8, oct = g % 8;
    if (!flag[g]) {
        child[8 * b + oct] = -1;
        return;
    }
    int c = next_off + pos[g];
    child[8 * b + oct] = c;
    int cx = 2 * coord[3 * b] + ((oct >> 2) & 1);
    int cy = 2 * coord[3 * b + 1] + ((oct >> 1) & 1);
    int cz = 2 * coord[3 * b + 2] + (oct & 1);
    lvl[c] = level + 1;
    coord[3 * c] = cx;
    coord[3 * c + 1] = cy;
    coord[3 * c + 2] = cz;
    parent[c] = b;
    code[c] = code[b] * 8 + oct;
    for (int k = 0; k < 4; ++k) rng[4 * c + k] = crng[4 * g + k];
    ctr[3 * c] = x0 + (cx + 0.5) * child_cell;
    ctr[3 * c + 1] = y0 + (cy + 0.5) * child_cell;
    ctr[3 * c + 2] = z0 + (cz + 0.5) * child_cell;
    for (int k = 0; k < 8; ++k) child[8 * c + k] = -1;
}

// Forest set-up: bounding box of each instance (one block per instance), then every
// point shifted by its instance's translation into the grid cell it owns.
__global__ void k_inst_bbox(const double* __restrict__ xyz, int64_t n, const int64_t* __restrict__ off,
                            double* __restrict__ out) {
    __shared__ double red[6][128];
    const int i = blockIdx.x;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t k = off[i] + threadIdx.x; k < off[i + 1]; k += blockDim.x)
        for (int d = 0; d < 3; ++d) {
            const double v = xyz[d * n + k];
            lo[d] = fmin(lo[d], v);
            hi[d] = fmax(hi[d], v);
        }
    for (int d = 0; d < 3; ++d) {
        red[d][threadIdx.x] = lo[d];
        red[3 + d][threadIdx.x] = hi[d];
    }
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int d = 0; d < 3; ++d) {
                red[d][threadIdx.x] = fmin(red[d][threadIdx.x], red[d][threadIdx.x + o]);
                red[3 + d][threadIdx.x] = fmax(red[3 + d][threadIdx.x], red[3 + d][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) out[6 * i + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void k_inst_shift(const double* __restrict__ xyz, int64_t n, const int64_t* __restrict__ off,
                             int ninst, const double* __restrict__ shift, double* __restrict__ out) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    int lo = 0, hi = ninst;                 // instance i with off[i] <= k < off[i + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= k) lo = mid;
        else hi = mid;
    }
    for (int d = 0; d < 3; ++d) out[d * n + k] = xyz[d * n + k] + shift[3 * lo + d];
}

struct ListCtx {
    LevelTable lt;
    int forest_level;                   // -1: one instance; else instances own the boxes of this level
    const int* lvl;
    const int* coord;
    const int* parent;
    const int* child;
    const int* leaf;
    const uint64_t* code;
    const int64_t* rng;
};

__device__ inline int find_box(const ListCtx& c, int level, int x, int y, int z) {
    int side = 1 << level;
    if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side) return -1;
    uint64_t key = morton3(x, y, z);
    int lo = c.lt.off[level], hi = c.lt.off[level + 1];
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (c.code[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < c.lt.off[level + 1] && c.code[lo] == key) ? lo : -1;
}

// Closed boxes touch or overlap.
__device__ inline bool adjacent(const ListCtx& c, int a, int b) {
    int la = c.lvl[a], lb = c.lvl[b];
    int L = max(la, lb);
    for (int d = 0; d < 3; ++d) {
        long long loa = (long long)c.coord[3 * a + d] << (L - la);
        long long hia = (long long)(c.coord[3 * a + d] + 1) << (L - la);
        long long lob = (long long)c.coord[3 * b + d] << (L - lb);
        long long hib = (long long)(c.coord[3 * b + d] + 1) << (L - lb);
        if (loa > hib || lob > hia) return false;
    }
    return true;
}

// Same instance: both boxes lie under one box of the forest level (always true for a
// single-instance tree; boxes above the forest level belong to no instance).
__device__ inline bool same_inst(const ListCtx& c, int a, int b) {
    if (c.forest_level < 0) return true;
    int la = c.lvl[a], lb = c.lvl[b];
    if (la < c.forest_level || lb < c.forest_level) return false;
    return (c.code[a] >> (3 * (la - c.forest_level))) == (c.code[b] >> (3 * (lb - c.forest_level)));
}

__device__ inline bool has_src(const ListCtx& c, int b) { return c.rng[4 * b + 1] > c.rng[4 * b]; }
__device__ inline bool has_trg(const ListCtx& c, int b) { return c.rng[4 * b + 3] > c.rng[4 * b + 2]; }

struct ListOut {
    int* cnt[4];
    const int* off[4];
    int* idx[4];
};

// mode 0: count into cnt; mode 1: write idx at off.
__global__ void k_lists(ListCtx c, int nbox, int mode, ListOut o, int* err) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    int n[4] = {0, 0, 0, 0};
    auto emit = [&](int which, int a) {
        if (mode == 1) o.idx[which][o.off[which][b] + n[which]] = a;
        ++n[which];
    };
    int l = c.lvl[b];
    int bx = c.coord[3 * b], by = c.coord[3 * b + 1], bz = c.coord[3 * b + 2];
    if (has_trg(c, b) && l >= c.forest_level) {
        // V list
        if (l >= 2) {
            int p = c.parent[b];
            int px = c.coord[3 * p], py = c.coord[3 * p + 1], pz = c.coord[3 * p + 2];
            for (int dx = -1; dx <= 1; ++dx)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dz = -1; dz <= 1; ++dz) {
                        int C = find_box(c, l - 1, px + dx, py + dy, pz + dz);
                        if (C < 0 || c.leaf[C] || !same_inst(c, C, b)) continue;
                        for (int k = 0; k < 8; ++k) {
                            int A = c.child[8 * C + k];
                            if (A < 0 || !has_src(c, A)) continue;
                            int ex = abs(c.coord[3 * A] - bx), ey = abs(c.coord[3 * A + 1] - by),
                                ez = abs(c.coord[3 * A + 2] - bz);
                            if (max(ex, max(ey, ez)) > 1) emit(1, A);
                        }
                    }
        }
        // X list: coarser-or-equal leaves adjacent to parent(B), not adjacent to B
        if (l >= 1) {
            int p = c.parent[b];
            for (int lp = l - 1; lp >= 0; --lp) {
                int sh = l - lp;
                int ax = bx >> sh, ay = by >> sh, az = bz >> sh;
                for (int dx = -1; dx <= 1; ++dx)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dz = -1; dz <= 1; ++dz) {
                            if (!dx && !dy && !dz) continue;
                            int A = find_box(c, lp, ax + dx, ay + dy, az + dz);
                            if (A < 0 || !c.leaf[A] || !has_src(c, A) || !same_inst(c, A, b)) continue;
                            if (adjacent(c, A, p) && !adjacent(c, A, b)) emit(3, A);
                        }
            }
        }
        if (c.leaf[b]) {
            // U and W: same-level colleagues and their descendants
            int stack[256];
            int sp = 0;
            for (int dx = -1; dx <= 1; ++dx)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dz = -1; dz <= 1; ++dz) {
                        int C = find_box(c, l, bx + dx, by + dy, bz + dz);
                        if (C < 0 || !same_inst(c, C, b)) continue;
                        if (c.leaf[C]) {
                            if (has_src(c, C)) emit(0, C);
                        } else {
                            for (int k = 0; k < 8; ++k) {
                                int D = c.child[8 * C + k];
                                if (D >= 0) {
                                    if (sp < 256) stack[sp++] = D;
                                    else atomicExch(err, 1);
                                }
                            }
                        }
                    }
            while (sp > 0) {
                int D = stack[--sp];
                if (!has_src(c, D)) continue;
                if (adjacent(c, D, b)) {
                    if (c.leaf[D]) {
                        emit(0, D);
                    } else {
                        for (int k = 0; k < 8; ++k) {
                            int E = c.child[8 * D + k];
                            if (E >= 0) {
                                if (sp < 256) stack[sp++] = E;
                                else atomicExch(err, 1);
                            }
                        }
                    }
                } else {
                    emit(2, D);
                }
            }
            // coarser leaves adjacent to B
            for (int lp = l - 1; lp >= 0; --lp) {
                int sh = l - lp;
                int ax = bx >> sh, ay = by >> sh, az = bz >> sh;
                for (int dx = -1; dx <= 1; ++dx)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dz = -1; dz <= 1; ++dz) {
                            if (!dx && !dy && !dz) continue;
                            int A = find_box(c, lp, ax + dx, ay + dy, az + dz);
                            if (A < 0 || !c.leaf[A] || !has_src(c, A) || !same_inst(c, A, b)) continue;
                            if (adjacent(c, A, b)) emit(0, A);
                        }
            }
        }
    }
    if (mode == 0)
        for (int k = 0; k < 4; ++k) o.cnt[k][b] = n[k];
}

template <typename T>
int grow(DBuf<T>& b, size_t need, size_t keep, cudaStream_t s) {
    if (need <= b.n) return KIFMM_OK;
    size_t cap = std::max(need, b.n * 2);
    T* np = nullptr;
    cudaError_t e = cudaMalloc((void**)&np, cap * sizeof(T));
    if (e != cudaSuccess) {
        set_error("cudaMalloc(%zu bytes): %s", cap * sizeof(T), cudaGetErrorString(e));
        return KIFMM_ERR_OOM;
    }
    if (keep) KF_CHECK_CUDA(cudaMemcpyAsync(np, b.p, keep * sizeof(T), cudaMemcpyDeviceToDevice, s));
    KF_CHECK_CUDA(cudaStreamSynchronize(s));
    if (b.p) cudaFree(b.p);
    b.p = np;
    b.n = cap;
    return KIFMM_OK;
}

int exclusive_scan_int(const int* in, int* out, int n, cudaStream_t s, DBuf<uint8_t>& tmp) {
    size_t bytes = 0;
    KF_CHECK_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, n, s));
    if (bytes > tmp.n) KF_TRY(tmp.alloc(bytes));
    KF_CHECK_CUDA(cub::DeviceScan::ExclusiveSum(tmp.p, bytes, in, out, n, s));
    return KIFMM_OK;
}

int sort_points(const double* xyz, int64_t n, const double lo[3], double inv_cell,
                DBuf<uint64_t>& key, DBuf<int64_t>& perm, DBuf<double>& sorted,
                cudaStream_t s) {
    DBuf<uint64_t> k0;
    DBuf<int64_t> i0;
    KF_TRY(k0.alloc(n));
    KF_TRY(i0.alloc(n));
    KF_TRY(key.alloc(n));
    KF_TRY(perm.alloc(n));
    KF_TRY(sorted.alloc(3 * n));
    k_morton<<<div_up(n, 256), 256, 0, s>>>(xyz, n, lo[0], lo[1], lo[2], inv_cell, k0.p, i0.p);
    KF_CHECK_LAUNCH();
    size_t bytes = 0;
    KF_CHECK_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, k0.p, key.p, i0.p, perm.p,
                                                  (int64_t)n, 0, 3 * kKeyBits, s));
    DBuf<uint8_t> tmp;
    KF_TRY(tmp.alloc(bytes));
    KF_CHECK_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, bytes, k0.p, key.p, i0.p, perm.p,
                                                  (int64_t)n, 0, 3 * kKeyBits, s));
    k_gather_xyz<<<div_up(n, 256), 256, 0, s>>>(xyz, perm.p, n, sorted.p);
    KF_CHECK_LAUNCH();
    KF_CHECK_CUDA(cudaStreamSynchronize(s));
    return KIFMM_OK;
}

int bbox(const double* xyz, int64_t n, double lo[3], double hi[3], cudaStream_t s) {
    int nb = (int)std::min<int64_t>(1024, std::max<int64_t>(1, div_up(n, 256)));
    DBuf<double> part;
    KF_TRY(part.alloc(6 * nb));
    k_bbox_partial<<<nb, 256, 0, s>>>(xyz, n, part.p);
    KF_CHECK_LAUNCH();
    std::vector<double> h;
    KF_TRY(download(h, part.p, 6 * nb, s));
    for (int b = 0; b < nb; ++b)
        for (int d = 0; d < 3; ++d) {
            double a = h[6 * b + d];
            if (std::isnan(a)) {
                set_error("invalid argument: non-finite coordinate");
                return KIFMM_ERR_INVALID_ARG;
            }
            lo[d] = std::min(lo[d], a);
            hi[d] = std::max(hi[d], h[6 * b + 3 + d]);
        }
    return KIFMM_OK;
}

// root_c / root_h: an explicit root cube (a forest's grid), or NULL to enclose the
// points; forest_level: the level whose boxes are the instances (-1: one instance).
int build(Tree& T, const double* src, int64_t ns, const double* trg, int64_t nt, int max_leaf,
          cudaStream_t s, const double* root_c = nullptr, double root_h = 0, int forest_level = -1) {
    T.ns = ns;
    T.same = (trg == nullptr);
    T.nt = T.same ? ns : nt;
    T.max_leaf = max_leaf;
    T.forest_level = forest_level;
    if (root_c) {
        for (int d = 0; d < 3; ++d) T.root_c[d] = root_c[d];
        T.root_h = root_h;
    } else {
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        KF_TRY(bbox(src, ns, lo, hi, s));
        if (!T.same) KF_TRY(bbox(trg, nt, lo, hi, s));
        double ext = 0;
        for (int d = 0; d < 3; ++d) {
            T.root_c[d] = 0.5 * (lo[d] + hi[d]);
            ext = std::max(ext, hi[d] - lo[d]);
        }
        if (ext <= 0) ext = 1.0;
        T.root_h = 0.5 * ext * (1.0 + 1e-6);
    }
    double x0[3] = {T.root_c[0] - T.root_h, T.root_c[1] - T.root_h, T.root_c[2] - T.root_h};
    double inv_cell = (double)(1u << kKeyBits) / (2.0 * T.root_h);

    KF_TRY(sort_points(src, ns, x0, inv_cell, T.skey, T.sperm, T.sxyz, s));
    if (!T.same) KF_TRY(sort_points(trg, T.nt, x0, inv_cell, T.tkey, T.tperm, T.txyz, s));
    const uint64_t* tkey = T.same ? T.skey.p : T.tkey.p;

    // level-by-level split
    size_t cap = 1024 + 16 * (size_t)((ns + T.nt) / std::max(1, max_leaf));
    KF_TRY(T.lvl.alloc(cap));
    KF_TRY(T.coord.alloc(3 * cap));
    KF_TRY(T.parent.alloc(cap));
    KF_TRY(T.child.alloc(8 * cap));
    KF_TRY(T.leaf.alloc(cap));
    KF_TRY(T.code.alloc(cap));
    KF_TRY(T.rng.alloc(4 * cap));
    KF_TRY(T.ctr.alloc(3 * cap));
    {
        int zero3[3] = {0, 0, 0};
        int one = 0, mone = -1;
        uint64_t c0 = 0;
        int64_t r0[4] = {0, ns, 0, T.nt};
        std::vector<int> ch(8, -1);
        KF_CHECK_CUDA(cudaMemcpyAsync(T.lvl.p, &one, sizeof(int), cudaMemcpyHostToDevice, s));
        KF_CHECK_CUDA(cudaMemcpyAsync(T.coord.p, zero3, 3 * sizeof(int), cudaMemcpyHostToDevice, s));
        KF_CHECK_CUDA(cudaMemcpyAsync(T.parent.p, &mone, sizeof(int), cudaMemcpyHostToDevice, s));
        KF_CHECK_CUDA(cudaMemcpyAsync(T.child.p, ch.data(), 8 * sizeof(int), cudaMemcpyHostToDevice, s));
        KF_CHECK_CUDA(cudaMemcpyAsync(T.code.p, &c0, sizeof(uint64_t), cudaMemcpyHostToDevice, s));
        KF_CHECK_CUDA(cudaMemcpyAsync(T.rng.p, r0, 4 * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        KF_CHECK_CUDA(cudaMemcpyAsync(T.ctr.p, T.root_c, 3 * sizeof(double), cudaMemcpyHostToDevice, s));
        KF_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    T.level_off.assign(1, 0);
    T.level_off.push_back(1);
    DBuf<int> flag, pos;
    DBuf<int64_t> crng;
    DBuf<uint8_t> tmp;
    for (int l = 0;; ++l) {
        int off = T.level_off[l], nl = T.level_off[l + 1] - off;
        KF_TRY(grow(flag, 8 * (size_t)nl, 0, s));
        KF_TRY(grow(pos, 8 * (size_t)nl, 0, s));
        KF_TRY(grow(crng, 32 * (size_t)nl, 0, s));
        int g = 8 * nl;
        k_split_count<<<div_up(g, 256), 256, 0, s>>>(off, nl, l, max_leaf, forest_level, T.same, T.skey.p, tkey,
                                                      T.code.p, T.rng.p, T.leaf.p, flag.p, crng.p);
        KF_CHECK_LAUNCH();
        KF_TRY(exclusive_scan_int(flag.p, pos.p, g, s, tmp));
        int last_pos = 0, last_flag = 0;
        KF_CHECK_CUDA(cudaMemcpyAsync(&last_pos, pos.p + g - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        KF_CHECK_CUDA(cudaMemcpyAsync(&last_flag, flag.p + g - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        KF_CHECK_CUDA(cudaStreamSynchronize(s));
        int nchild = last_pos + last_flag;
        int next_off = off + nl;
        size_t need = (size_t)next_off + nchild;
        size_t keep = next_off;
        KF_TRY(grow(T.lvl, need, keep, s));
        KF_TRY(grow(T.coord, 3 * need, 3 * keep, s));
        KF_TRY(grow(T.parent, need, keep, s));
        KF_TRY(grow(T.child, 8 * need, 8 * keep, s));
        KF_TRY(grow(T.leaf, need, keep, s));
        KF_TRY(grow(T.code, need, keep, s));
        KF_TRY(grow(T.rng, 4 * need, 4 * keep, s));
        KF_TRY(grow(T.ctr, 3 * need, 3 * keep, s));
        double child_cell = 2.0 * T.root_h / (double)(1 << (l + 1));
        k_split_emit<<<div_up(g, 256), 256, 0, s>>>(off, nl, l, next_off, flag.p, pos.p, crng.p,
                                                     x0[0], x0[1], x0[2], child_cell, T.lvl.p,
                                                     T.coord.p, T.parent.p, T.child.p, T.code.p,
                                                     T.rng.p, T.ctr.p);
        KF_CHECK_LAUNCH();
        if (nchild == 0) break;
        T.level_off.push_back(next_off + nchild);
    }
    T.nlev = (int)T.level_off.size() - 1;
    T.nbox = T.level_off.back();
    T.level_half.resize(T.nlev);
    for (int l = 0; l < T.nlev; ++l) T.level_half[l] = T.root_h / (double)(1 << l);

    // interaction lists: count, scan, fill
    ListCtx c;
    memset(&c.lt, 0, sizeof(c.lt));
    for (int l = 0; l <= T.nlev; ++l) c.lt.off[l] = T.level_off[l];
    for (int l = T.nlev + 1; l < kMaxDepth + 3; ++l) c.lt.off[l] = T.nbox;
    c.lt.nlev = T.nlev;
    c.forest_level = forest_level;
    c.lvl = T.lvl.p;
    c.coord = T.coord.p;
    c.parent = T.parent.p;
    c.child = T.child.p;
    c.leaf = T.leaf.p;
    c.code = T.code.p;
    c.rng = T.rng.p;
    DBuf<int> cnt[4];
    DBuf<int>* offs[4] = {&T.u_off, &T.v_off, &T.w_off, &T.x_off};
    DBuf<int>* idxs[4] = {&T.u_idx, &T.v_idx, &T.w_idx, &T.x_idx};
    ListOut o;
    for (int k = 0; k < 4; ++k) {
        KF_TRY(cnt[k].alloc(T.nbox + 1));
        KF_CHECK_CUDA(cudaMemsetAsync(cnt[k].p, 0, (T.nbox + 1) * sizeof(int), s));
        KF_TRY(offs[k]->alloc(T.nbox + 1));
        o.cnt[k] = cnt[k].p;
        o.off[k] = offs[k]->p;
        o.idx[k] = nullptr;
    }
    DBuf<int> err;
    KF_TRY(err.alloc(1));
    KF_CHECK_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    k_lists<<<div_up(T.nbox, 128), 128, 0, s>>>(c, T.nbox, 0, o, err.p);
    KF_CHECK_LAUNCH();
    int64_t tot[4];
    for (int k = 0; k < 4; ++k) {
        KF_TRY(exclusive_scan_int(cnt[k].p, offs[k]->p, T.nbox + 1, s, tmp));
        int t = 0;
        KF_CHECK_CUDA(cudaMemcpyAsync(&t, offs[k]->p + T.nbox, sizeof(int), cudaMemcpyDeviceToHost, s));
        KF_CHECK_CUDA(cudaStreamSynchronize(s));
        tot[k] = t;
        KF_TRY(idxs[k]->alloc(std::max<int64_t>(1, t)));
        o.idx[k] = idxs[k]->p;
    }
    k_lists<<<div_up(T.nbox, 128), 128, 0, s>>>(c, T.nbox, 1, o, err.p);
    KF_CHECK_LAUNCH();
    int herr = 0;
    KF_CHECK_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    KF_CHECK_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        set_error("interaction-list traversal stack overflow");
        return KIFMM_ERR_UNSUPPORTED;
    }
    T.nu = tot[0];
    T.nv = tot[1];
    T.nw = tot[2];
    T.nx = tot[3];

    // host copies for plan construction and export
    KF_TRY(download(T.h_lvl, T.lvl.p, T.nbox, s));
    KF_TRY(download(T.h_parent, T.parent.p, T.nbox, s));
    KF_TRY(download(T.h_leaf, T.leaf.p, T.nbox, s));
    KF_TRY(download(T.h_coord, T.coord.p, 3 * (size_t)T.nbox, s));
    KF_TRY(download(T.h_child, T.child.p, 8 * (size_t)T.nbox, s));
    KF_TRY(download(T.h_rng, T.rng.p, 4 * (size_t)T.nbox, s));
    KF_TRY(download(T.h_ctr, T.ctr.p, 3 * (size_t)T.nbox, s));
    KF_TRY(download(T.h_u_off, T.u_off.p, T.nbox + 1, s));
    KF_TRY(download(T.h_u_idx, T.u_idx.p, T.nu, s));
    KF_TRY(download(T.h_v_off, T.v_off.p, T.nbox + 1, s));
    KF_TRY(download(T.h_v_idx, T.v_idx.p, T.nv, s));
    KF_TRY(download(T.h_w_off, T.w_off.p, T.nbox + 1, s));
    KF_TRY(download(T.h_w_idx, T.w_idx.p, T.nw, s));
    KF_TRY(download(T.h_x_off, T.x_off.p, T.nbox + 1, s));
    KF_TRY(download(T.h_x_idx, T.x_idx.p, T.nx, s));
    T.nleaf = 0;
    T.p2p_pairs = 0;
    for (int b = 0; b < T.nbox; ++b) {
        if (!T.h_leaf[b]) continue;
        ++T.nleaf;
        int64_t ntb = T.h_rng[4 * b + 3] - T.h_rng[4 * b + 2];
        int64_t srcs = 0;
        for (int k = T.h_u_off[b]; k < T.h_u_off[b + 1]; ++k) {
            int a = T.h_u_idx[k];
            srcs += T.h_rng[4 * a + 1] - T.h_rng[4 * a];
        }
        for (int k = T.h_w_off[b]; k < T.h_w_off[b + 1]; ++k) {
            int a = T.h_w_idx[k];
            srcs += T.h_rng[4 * a + 1] - T.h_rng[4 * a];
        }
        T.p2p_pairs += ntb * srcs;
    }
    return KIFMM_OK;
}

// Forest of independent instances (sources = targets): instance i's points are
// translated, unscaled, into cell i (Morton order) of a 2^L x 2^L x 2^L grid whose cells
// are as wide as the widest instance (plus a margin); the octree over the grid has the
// cells as its level-L boxes and its lists never cross cells, so every FMM phase runs
// once for all instances and no instance sees another.
int build_forest(Tree& T, const double* xyz, int64_t n, const int64_t* h_off, int ninst, int max_leaf,
                 cudaStream_t s) {
    int L = 0;
    while ((1LL << (3 * L)) < ninst) ++L;
    DBuf<int64_t> off;
    DBuf<double> bb, shift, moved;
    KF_TRY(off.alloc(ninst + 1));
    KF_TRY(bb.alloc(6 * (size_t)ninst));
    KF_TRY(shift.alloc(3 * (size_t)ninst));
    KF_TRY(moved.alloc(3 * (size_t)n));
    KF_CHECK_CUDA(cudaMemcpyAsync(off.p, h_off, (ninst + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    k_inst_bbox<<<ninst, 128, 0, s>>>(xyz, n, off.p, bb.p);
    KF_CHECK_LAUNCH();
    std::vector<double> h_bb(6 * (size_t)ninst), h_shift(3 * (size_t)ninst);
    KF_CHECK_CUDA(cudaMemcpyAsync(h_bb.data(), bb.p, h_bb.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    KF_CHECK_CUDA(cudaStreamSynchronize(s));
    double ext = 0;
    for (int i = 0; i < ninst; ++i)
        for (int d = 0; d < 3; ++d) {
            if (!(h_bb[6 * i + d] <= h_bb[6 * i + 3 + d])) {
                set_error("instance %d has non-finite coordinates", i);
                return KIFMM_ERR_INVALID_ARG;
            }
            ext = std::max(ext, h_bb[6 * i + 3 + d] - h_bb[6 * i + d]);
        }
    const double cell = (ext > 0 ? ext : 1.0) * 1.01;   // every instance strictly inside its cell
    for (int i = 0; i < ninst; ++i) {
        int c[3] = {0, 0, 0};
        for (int k = 0; k < L; ++k) {
            c[0] |= ((i >> (3 * k + 2)) & 1) << k;
            c[1] |= ((i >> (3 * k + 1)) & 1) << k;
            c[2] |= ((i >> (3 * k)) & 1) << k;
        }
        for (int d = 0; d < 3; ++d)
            h_shift[3 * i + d] = (c[d] + 0.5) * cell - 0.5 * (h_bb[6 * i + d] + h_bb[6 * i + 3 + d]);
    }
    KF_CHECK_CUDA(cudaMemcpyAsync(shift.p, h_shift.data(), h_shift.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    k_inst_shift<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xyz, n, off.p, ninst, shift.p, moved.p);
    KF_CHECK_LAUNCH();
    const double half = 0.5 * cell * (double)(1 << L);
    const double rc[3] = {half, half, half};
    KF_TRY(build(T, moved.p, n, nullptr, 0, max_leaf, s, rc, half, L));
    T.inst_off.assign(h_off, h_off + ninst + 1);
    KF_CHECK_CUDA(cudaStreamSynchronize(s));   // the translated copy is freed on return
    return KIFMM_OK;
}

}  // namespace

}  // namespace kifmm

using namespace kifmm;

extern "C" int kifmm_tree_build(const double* src_xyz, int64_t n_src, const double* trg_xyz,
                                int64_t n_trg, int max_leaf, void* stream, kifmm_tree* out) {
    clear_error();
    KF_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    KF_ARG(src_xyz != nullptr, "src_xyz is NULL");
    KF_ARG(n_src >= 1 && n_src < (1LL << 31), "n_src must be in [1, 2^31)");
    KF_ARG(trg_xyz == nullptr || (n_trg >= 1 && n_trg < (1LL << 31)), "n_trg must be in [1, 2^31)");
    KF_ARG(max_leaf >= 1 && max_leaf <= 1024, "max_leaf must be in [1, 1024]");
    cudaStream_t s = (cudaStream_t)stream;
    kifmm_tree t = new (std::nothrow) kifmm_tree_s;
    if (!t) {
        set_error("host allocation failed");
        return KIFMM_ERR_OOM;
    }
    cudaGetDevice(&t->t.device);
    int rc = build(t->t, src_xyz, n_src, trg_xyz, n_trg, max_leaf, s);
    if (rc != KIFMM_OK) {
        delete t;
        return rc;
    }
    *out = t;
    return KIFMM_OK;
}

extern "C" int kifmm_forest_build(const double* xyz, int64_t n, const int64_t* inst_off, int n_inst,
                                  int max_leaf, void* stream, kifmm_tree* out) {
    clear_error();
    KF_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    KF_ARG(xyz != nullptr && inst_off != nullptr, "xyz or inst_off is NULL");
    KF_ARG(n >= 1 && n < (1LL << 31), "n must be in [1, 2^31)");
    KF_ARG(n_inst >= 1 && n_inst <= KIFMM_MAX_INSTANCES, "n_inst must be in [1, KIFMM_MAX_INSTANCES]");
    KF_ARG(max_leaf >= 1 && max_leaf <= 1024, "max_leaf must be in [1, 1024]");
    KF_ARG(inst_off[0] == 0 && inst_off[n_inst] == n, "inst_off must run from 0 to n");
    for (int i = 0; i < n_inst; ++i) KF_ARG(inst_off[i + 1] > inst_off[i], "every instance needs a point");
    cudaStream_t s = (cudaStream_t)stream;
    kifmm_tree t = new (std::nothrow) kifmm_tree_s;
    if (!t) {
        set_error("host allocation failed");
        return KIFMM_ERR_OOM;
    }
    cudaGetDevice(&t->t.device);
    int rc = build_forest(t->t, xyz, n, inst_off, n_inst, max_leaf, s);
    if (rc != KIFMM_OK) {
        delete t;
        return rc;
    }
    *out = t;
    return KIFMM_OK;
}

extern "C" int kifmm_tree_get_stats(kifmm_tree tree, kifmm_tree_stats* st) {
    clear_error();
    KF_ARG(tree && st, "NULL handle or stats");
    const Tree& T = tree->t;
    st->n_src = T.ns;
    st->n_trg = T.nt;
    st->n_boxes = T.nbox;
    st->n_leaves = T.nleaf;
    st->n_levels = T.nlev;
    st->max_leaf = T.max_leaf;
    st->n_u = T.nu;
    st->n_v = T.nv;
    st->n_w = T.nw;
    st->n_x = T.nx;
    st->p2p_pairs = T.p2p_pairs;
    for (int d = 0; d < 3; ++d) st->root_center[d] = T.root_c[d];
    st->root_half = T.root_h;
    st->n_instances = T.forest_level < 0 ? 1 : (int32_t)(T.inst_off.size() - 1);
    st->forest_level = T.forest_level;
    return KIFMM_OK;
}

extern "C" int kifmm_tree_export(kifmm_tree tree, int32_t* box_level, int32_t* box_coord,
                                 int32_t* box_parent, int32_t* box_leaf, int64_t* box_range,
                                 int64_t* src_perm, int64_t* trg_perm) {
    clear_error();
    KF_ARG(tree, "NULL handle");
    const Tree& T = tree->t;
    if (box_level) std::copy(T.h_lvl.begin(), T.h_lvl.end(), box_level);
    if (box_coord) std::copy(T.h_coord.begin(), T.h_coord.end(), box_coord);
    if (box_parent) std::copy(T.h_parent.begin(), T.h_parent.end(), box_parent);
    if (box_leaf) std::copy(T.h_leaf.begin(), T.h_leaf.end(), box_leaf);
    if (box_range) std::copy(T.h_rng.begin(), T.h_rng.end(), box_range);
    if (src_perm) KF_CHECK_CUDA(cudaMemcpy(src_perm, T.sperm.p, T.ns * sizeof(int64_t), cudaMemcpyDeviceToHost));
    if (trg_perm) {
        const int64_t* p = T.same ? T.sperm.p : T.tperm.p;
        KF_CHECK_CUDA(cudaMemcpy(trg_perm, p, T.nt * sizeof(int64_t), cudaMemcpyDeviceToHost));
    }
    return KIFMM_OK;
}

extern "C" int kifmm_tree_export_list(kifmm_tree tree, int which, int64_t* offsets, int32_t* idx) {
    clear_error();
    KF_ARG(tree, "NULL handle");
    KF_ARG(which >= 0 && which <= 3, "which must be KIFMM_LIST_U/V/W/X");
    const Tree& T = tree->t;
    const std::vector<int>* off[4] = {&T.h_u_off, &T.h_v_off, &T.h_w_off, &T.h_x_off};
    const std::vector<int>* ix[4] = {&T.h_u_idx, &T.h_v_idx, &T.h_w_idx, &T.h_x_idx};
    if (offsets)
        for (int b = 0; b <= T.nbox; ++b) offsets[b] = (*off[which])[b];
    if (idx) std::copy(ix[which]->begin(), ix[which]->end(), idx);
    return KIFMM_OK;
}

extern "C" int kifmm_tree_destroy(kifmm_tree tree) {
    clear_error();
    delete tree;
    return KIFMM_OK;
}
