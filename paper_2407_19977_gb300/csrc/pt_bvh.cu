// pt_bvh.cu -- device BVH build (Sec. 5.1.1: AABB hierarchy over the triangles).
//
// 1. centroid bounds, 2. 63-bit Morton codes, 3. LSD radix sort (8 passes of 8 bits),
// 4. binary radix tree over the sorted codes (Karras, HPG 2012), 5. bottom-up boxes,
// 6. top-down collapse into a wide BVH with 8-bit quantised child boxes (80-byte nodes of 8
//    child slots, at most max_width of them used; the layout of compressed wide BVHs, Ylitie,
//    Karras, Laine, HPG 2017), whose leaf triangles are laid out contiguously per node.
// The environment's sampling tables (marginal/conditional CDFs) are built here too.
#include <vector>

#include "pt_internal.h"

#define LEAF_BIT 0x80000000u

__device__ __forceinline__ uint32_t f2ord_b(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f_b(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__device__ __forceinline__ float3 tri_centroid(const float4* t, uint32_t i) {
    const float4 a = t[3u * i], b = t[3u * i + 1], c = t[3u * i + 2];
    return mk3((a.x + b.x + c.x) * (1.0f / 3.0f), (a.y + b.y + c.y) * (1.0f / 3.0f), (a.z + b.z + c.z) * (1.0f / 3.0f));
}

__global__ void k_centroid_bounds(const float4* tris, uint32_t n, uint32_t* cb) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
    if (i < n) {
        const float3 c = tri_centroid(tris, i);
        lo[0] = hi[0] = c.x; lo[1] = hi[1] = c.y; lo[2] = hi[2] = c.z;
    }
    for (int a = 0; a < 3; ++a) {
        for (int off = 16; off > 0; off >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int a = 0; a < 3; ++a) {
            atomicMin(&cb[a], f2ord_b(lo[a]));
            atomicMax(&cb[3 + a], f2ord_b(hi[a]));
        }
    }
}

__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;  // 21 bits
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

__global__ void k_morton(const float4* tris, uint32_t n, const uint32_t* cb, uint64_t* keys, uint32_t* vals) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float3 c = tri_centroid(tris, i);
    float q[3];
    for (int a = 0; a < 3; ++a) {
        const float lo = ord2f_b(cb[a]), hi = ord2f_b(cb[3 + a]);
        const float ext = hi - lo;
        const float t = ext > 0.0f ? (comp3(c, a) - lo) / ext : 0.5f;
        q[a] = fminf(fmaxf(t * 2097152.0f, 0.0f), 2097151.0f);
    }
    keys[i] = spread3((uint32_t)q[0]) << 2 | spread3((uint32_t)q[1]) << 1 | spread3((uint32_t)q[2]);
    vals[i] = i;
}

// ------------------------------------------------------------------ LSD radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;

__global__ void k_rs_hist(const uint64_t* keys, uint32_t n, int shift, uint32_t* hist, uint32_t nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t base = blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const uint32_t idx = base + r * RS_THREADS + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of m counters by one block of 1024 threads
__global__ void k_rs_scan(uint32_t* data, uint32_t m) {
    __shared__ uint32_t part[1024];
    const uint32_t per = (m + 1023) / 1024;
    const uint32_t b = threadIdx.x * per, e = min(b + per, m);
    uint32_t sum = 0;
    for (uint32_t i = b; i < e; ++i) sum += data[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t v = threadIdx.x >= (uint32_t)off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - sum;
    for (uint32_t i = b; i < e; ++i) {
        const uint32_t v = data[i];
        data[i] = run;
        run += v;
    }
}

// stable scatter: tile order = round-major, then thread; ranks from warp match + per-warp counts
__global__ void k_rs_scatter(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout, uint32_t n,
                             int shift, const uint32_t* hist, uint32_t nblocks) {
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[RS_THREADS / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = hist[tid * nblocks + blockIdx.x];
    const uint32_t lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const uint32_t idx = blockIdx.x * RS_TILE + r * RS_THREADS + tid;
        const bool valid = idx < n;
        const uint64_t key = valid ? kin[idx] : 0ull;
        const uint32_t digit = valid ? (uint32_t)((key >> shift) & 255u) : 256u;
        for (int j = tid; j < (RS_THREADS / 32) * 256; j += RS_THREADS) (&wcnt[0][0])[j] = 0u;
        __syncthreads();
        const uint32_t peers = __match_any_sync(0xffffffffu, digit);
        const uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        {
            uint32_t run = base[tid];
            for (int w = 0; w < RS_THREADS / 32; ++w) {
                const uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = run;
                run += c;
            }
            base[tid] = run;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = wcnt[warp][digit] + rank;
            kout[pos] = key;
            vout[pos] = vin[idx];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ binary radix tree
__device__ __forceinline__ int lcp(const uint64_t* keys, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    const uint64_t a = keys[i], b = keys[j];
    if (a == b) return 64 + __clz((uint32_t)(i ^ j));
    return __clzll((long long)(a ^ b));
}

__global__ void k_karras(const uint64_t* keys, int n, uint32_t* left, uint32_t* right, uint32_t* par_int,
                         uint32_t* par_leaf, uint32_t* first, uint32_t* last) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = (lcp(keys, n, i, i + 1) - lcp(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = lcp(keys, n, i, i - d);
    int lmax = 2;
    while (lcp(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (lcp(keys, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = lcp(keys, n, i, j);
    int s = 0, t = l;
    for (;;) {
        t = (t + 1) >> 1;
        if (lcp(keys, n, i, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
    }
    const int gamma = i + s * d + min(d, 0);
    const int lo = min(i, j), hi = max(i, j);
    const uint32_t L = (lo == gamma) ? (LEAF_BIT | (uint32_t)gamma) : (uint32_t)gamma;
    const uint32_t R = (hi == gamma + 1) ? (LEAF_BIT | (uint32_t)(gamma + 1)) : (uint32_t)(gamma + 1);
    left[i] = L;
    right[i] = R;
    first[i] = (uint32_t)lo;
    last[i] = (uint32_t)hi;
    if (L & LEAF_BIT) par_leaf[L & ~LEAF_BIT] = (uint32_t)i; else par_int[L] = (uint32_t)i;
    if (R & LEAF_BIT) par_leaf[R & ~LEAF_BIT] = (uint32_t)i; else par_int[R] = (uint32_t)i;
    if (i == 0) par_int[0] = 0xffffffffu;
}

struct Box {
    float3 lo, hi;
};

__device__ __forceinline__ Box tri_box(const float4* tris, uint32_t t) {
    const float4 a = tris[3u * t], b = tris[3u * t + 1], c = tris[3u * t + 2];
    Box r;
    r.lo = mk3(fminf(a.x, fminf(b.x, c.x)), fminf(a.y, fminf(b.y, c.y)), fminf(a.z, fminf(b.z, c.z)));
    r.hi = mk3(fmaxf(a.x, fmaxf(b.x, c.x)), fmaxf(a.y, fmaxf(b.y, c.y)), fmaxf(a.z, fmaxf(b.z, c.z)));
    return r;
}
__device__ __forceinline__ Box box_union(Box a, Box b) {
    Box r;
    r.lo = mk3(fminf(a.lo.x, b.lo.x), fminf(a.lo.y, b.lo.y), fminf(a.lo.z, b.lo.z));
    r.hi = mk3(fmaxf(a.hi.x, b.hi.x), fmaxf(a.hi.y, b.hi.y), fmaxf(a.hi.z, b.hi.z));
    return r;
}

// ---- cost-optimal collapse: per binary node, the least surface-area cost of its subtree
// when it fills exactly j = 1..8 slots of a wide node (the dynamic programme of Ylitie,
// Karras and Laine, HPG 2017, restated for leaves of at most leaf_size triangles and nodes of
// at most W = width children).  With A the (half) surface area, a wide node visit costing 1
// plus box_cost per slot and a triangle test tri_cost:
//   C(k)    = A(k) * tri_cost * count(k)                          if count(k) <= leaf_size
//           = A(k) + min_{j=2..W} E(k, j) + A(k) * box_cost * j    otherwise (a wide node)
//   E(k, 1) = C(k);  E(k, j) = min_{i=1..j-1} E(L, i) + E(R, j - i)  (j >= 2)
// and a single triangle costs A * tri_cost as one slot and cannot fill more.  dec[k] keeps
// the choices in nibbles: nibble 0 the slot count j of C(k) for a wide node, nibble j - 1
// (j = 2..8) the split i of E(k, j).
struct DpArrays {
    float* cost;            // 8 per binary node: E(k, 1..8); null: greedy collapse
    uint32_t* dec;          // choices, one word per binary node
    uint32_t leaf_size;
    float tri_cost, box_cost;
    uint32_t width;         // most children of a wide node, 2..8
};

__device__ __forceinline__ float half_area_box(float3 lo, float3 hi) {
    const float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return dx * dy + dy * dz + dz * dx;
}

// E(child, 1..8) of a child reference: a triangle (its area given) or a binary node
__device__ __forceinline__ void dp_child(const DpArrays& D, uint32_t ref, float leaf_area, float (&c)[8]) {
    if (ref & 0x80000000u) {
        c[0] = leaf_area * D.tri_cost;
#pragma unroll
        for (int j = 1; j < 8; ++j) c[j] = __int_as_float(0x7f800000);
    } else {
        const float4 a = __ldcg(reinterpret_cast<const float4*>(D.cost + 8u * ref));
        const float4 b = __ldcg(reinterpret_cast<const float4*>(D.cost + 8u * ref) + 1);
        c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w; c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
    }
}

__device__ __forceinline__ void dp_node(const DpArrays& D, uint32_t k, uint32_t lref, float larea, uint32_t rref,
                                        float rarea, uint32_t count, float area) {
    float cl[8], cr[8], e[8];
    dp_child(D, lref, larea, cl);
    dp_child(D, rref, rarea, cr);
    uint32_t dec = 0;
#pragma unroll
    for (uint32_t j = 2; j <= 8; ++j) {
        float best = __int_as_float(0x7f800000);
        uint32_t bi = 1;
        for (uint32_t i = 1; i < j; ++i) {
            const float v = cl[i - 1] + cr[j - i - 1];
            if (v < best) { best = v; bi = i; }
        }
        e[j - 1] = best;
        dec |= bi << (4 * (j - 1));
    }
    if (count <= D.leaf_size) {
        e[0] = area * D.tri_cost * (float)count;
    } else {
        float best = __int_as_float(0x7f800000);
        uint32_t bj = 2;
        for (uint32_t j = 2; j <= D.width; ++j) {
            const float v = e[j - 1] + area * D.box_cost * (float)j;
            if (v < best) { best = v; bj = j; }
        }
        e[0] = area + best;
        dec |= bj;
    }
    __stcg(reinterpret_cast<float4*>(D.cost + 8u * k), make_float4(e[0], e[1], e[2], e[3]));
    __stcg(reinterpret_cast<float4*>(D.cost + 8u * k) + 1, make_float4(e[4], e[5], e[6], e[7]));
    __stcg(D.dec + k, dec);
}

struct BinTree {
    const uint32_t *left, *right, *first, *last, *perm;
    float4 *blo, *bhi;
    const float4* tris;
};

__device__ __forceinline__ Box ref_box(const BinTree& T, uint32_t ref) {
    if (ref & LEAF_BIT) return tri_box(T.tris, T.perm[ref & ~LEAF_BIT]);
    const float4 lo = __ldcg(T.blo + ref), hi = __ldcg(T.bhi + ref);
    Box b;
    b.lo = xyz(lo);
    b.hi = xyz(hi);
    return b;
}

__global__ void k_bottom_up(BinTree T, int n, const uint32_t* par_int, const uint32_t* par_leaf, uint32_t* flags,
                            DpArrays D) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t node = par_leaf[i];
    while (node != 0xffffffffu) {
        __threadfence();
        if (atomicAdd(&flags[node], 1u) == 0u) return;  // first child to arrive stops
        __threadfence();
        const uint32_t l = T.left[node], r = T.right[node];
        const Box bl = ref_box(T, l), br = ref_box(T, r);
        const Box b = box_union(bl, br);
        __stcg(T.blo + node, make_float4(b.lo.x, b.lo.y, b.lo.z, 0.0f));
        __stcg(T.bhi + node, make_float4(b.hi.x, b.hi.y, b.hi.z, 0.0f));
        if (D.cost)
            dp_node(D, node, l, half_area_box(bl.lo, bl.hi), r, half_area_box(br.lo, br.hi),
                    T.last[node] - T.first[node] + 1u, half_area_box(b.lo, b.hi));
        node = par_int[node];
    }
}

// ------------------------------------------------------------------ PLOC binary tree
// Parallel locally-ordered clustering (Meister & Bittner, IEEE TVCG 2018): the clusters start
// as the triangles in Morton order; each round every cluster finds, within PLOC_R positions on
// either side, the cluster whose union with it has the least surface area, mutual pairs merge
// into a new binary node (at the lower position), and the survivors are compacted in order.
// Pairs are ranked by (area, lower index, higher index), a total order, so the globally least
// pair within the window is always mutual and every round merges at least once.  Merges get
// node indices counting down from n - 2, so the last merge (the root) is node 0, and every
// node's children have higher indices than the node.  A top-down pass over the rounds in
// reverse then lays the triangles out in tree order, giving each subtree the contiguous
// [first, last] range the collapse needs.
constexpr int PLOC_R = 16;
constexpr int PLOC_THREADS = 256;
constexpr int PLOC_SCAN_ITEMS = 4;                      // per thread of the block scan
constexpr int PLOC_SCAN_TILE = PLOC_THREADS * PLOC_SCAN_ITEMS;

struct Clusters {
    uint32_t* ref;      // LEAF_BIT | triangle id, or binary node index
    uint32_t* cnt;      // triangles below
    float4 *lo, *hi;    // bounds
};

__device__ __forceinline__ float half_area3(float3 lo, float3 hi) {
    const float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return dx * dy + dy * dz + dz * dx;
}

__global__ void k_ploc_init(const float4* tris, const uint32_t* perm, uint32_t n, Clusters c) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t t = perm[i];
    const Box b = tri_box(tris, t);
    c.ref[i] = LEAF_BIT | t;
    c.cnt[i] = 1u;
    c.lo[i] = make_float4(b.lo.x, b.lo.y, b.lo.z, 0.0f);
    c.hi[i] = make_float4(b.hi.x, b.hi.y, b.hi.z, 0.0f);
}

// nearest neighbour of each of the m clusters within the window (lowest index on equal area)
__global__ void __launch_bounds__(PLOC_THREADS) k_ploc_nn(Clusters c, uint32_t m, uint32_t* nn) {
    __shared__ float4 slo[PLOC_THREADS + 2 * PLOC_R], shi[PLOC_THREADS + 2 * PLOC_R];
    const int base = (int)(blockIdx.x * PLOC_THREADS) - PLOC_R;
    for (int k = threadIdx.x; k < PLOC_THREADS + 2 * PLOC_R; k += PLOC_THREADS) {
        const int g = base + k;
        if (g >= 0 && g < (int)m) { slo[k] = c.lo[g]; shi[k] = c.hi[g]; }
    }
    __syncthreads();
    const int i = (int)(blockIdx.x * PLOC_THREADS + threadIdx.x);
    if (i >= (int)m) return;
    const int li = threadIdx.x + PLOC_R;
    const float3 alo = xyz(slo[li]), ahi = xyz(shi[li]);
    float best = __int_as_float(0x7f800000);
    int bj = -1;
    const int j0 = max(i - PLOC_R, 0), j1 = min(i + PLOC_R, (int)m - 1);
    for (int j = j0; j <= j1; ++j) {
        if (j == i) continue;
        const int lj = j - base;
        const float3 blo = xyz(slo[lj]), bhi = xyz(shi[lj]);
        const float a = half_area3(mk3(fminf(alo.x, blo.x), fminf(alo.y, blo.y), fminf(alo.z, blo.z)),
                                   mk3(fmaxf(ahi.x, bhi.x), fmaxf(ahi.y, bhi.y), fmaxf(ahi.z, bhi.z)));
        if (a < best) { best = a; bj = j; }
    }
    nn[i] = (uint32_t)bj;
}

// per cluster: survives (1) and creates a node (bit 32) -- the lower index of a mutual pair --
// or is absorbed (0); exclusive block-level scan of those 64-bit values, block totals aside
__device__ __forceinline__ uint64_t ploc_flag(const uint32_t* nn, uint32_t m, uint32_t i) {
    if (i >= m) return 0ull;
    const uint32_t j = nn[i];
    if (j >= m) return 1ull;                       // m == 1: no neighbour
    if (nn[j] != i) return 1ull;
    return i < j ? ((1ull << 32) | 1ull) : 0ull;
}

__global__ void __launch_bounds__(PLOC_THREADS) k_ploc_scan(const uint32_t* nn, uint32_t m, uint64_t* pre,
                                                            uint64_t* block_sum) {
    __shared__ uint64_t warp_sum[PLOC_THREADS / 32];
    const uint32_t t0 = blockIdx.x * PLOC_SCAN_TILE + threadIdx.x * PLOC_SCAN_ITEMS;
    uint64_t v[PLOC_SCAN_ITEMS], run = 0;
#pragma unroll
    for (int k = 0; k < PLOC_SCAN_ITEMS; ++k) {
        v[k] = ploc_flag(nn, m, t0 + k);
        run += v[k];
    }
    // inclusive scan of the per-thread totals across the warp, then across warps
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = run;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    uint64_t before = 0;
    for (int w = 0; w < warp; ++w) before += warp_sum[w];
    uint64_t acc = before + x - run;               // exclusive prefix of this thread
#pragma unroll
    for (int k = 0; k < PLOC_SCAN_ITEMS; ++k) {
        if (t0 + k < m) pre[t0 + k] = acc;
        acc += v[k];
    }
    if (threadIdx.x == PLOC_THREADS - 1) block_sum[blockIdx.x] = before + x;
}

// exclusive scan of nb block totals by one block; the grand total goes to data[nb]
__global__ void k_ploc_scan_top(uint64_t* data, uint32_t nb) {
    __shared__ uint64_t part[1024];
    const uint32_t per = (nb + 1023) / 1024;
    const uint32_t b = threadIdx.x * per, e = min(b + per, nb);
    uint64_t sum = 0;
    for (uint32_t i = b; i < e; ++i) sum += data[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint64_t v = threadIdx.x >= (uint32_t)off ? part[threadIdx.x - off] : 0ull;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint64_t run = part[threadIdx.x] - sum;
    for (uint32_t i = b; i < e; ++i) {
        const uint64_t v = data[i];
        data[i] = run;
        run += v;
    }
    if (threadIdx.x == 1023) data[nb] = part[1023];
}

// survivors to their compacted position; a mutual pair becomes binary node
// n - 2 - (merged_before + its rank among this round's merges)
__global__ void k_ploc_compact(Clusters a, Clusters b, const uint32_t* nn, uint32_t m, const uint64_t* pre,
                               const uint64_t* block_pre, uint32_t n, uint32_t merged_before, uint32_t* left,
                               uint32_t* right, uint32_t* count, float4* blo, float4* bhi, DpArrays D) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint64_t f = ploc_flag(nn, m, i);
    if (f == 0ull) return;
    const uint64_t p = pre[i] + block_pre[i / PLOC_SCAN_TILE];
    const uint32_t pos = (uint32_t)(p & 0xffffffffull);
    if (f == 1ull) {
        b.ref[pos] = a.ref[i];
        b.cnt[pos] = a.cnt[i];
        b.lo[pos] = a.lo[i];
        b.hi[pos] = a.hi[i];
        return;
    }
    const uint32_t j = nn[i];
    const uint32_t node = n - 2u - (merged_before + (uint32_t)(p >> 32));
    const float4 l0 = a.lo[i], h0 = a.hi[i], l1 = a.lo[j], h1 = a.hi[j];
    const float4 lo = make_float4(fminf(l0.x, l1.x), fminf(l0.y, l1.y), fminf(l0.z, l1.z), 0.0f);
    const float4 hi = make_float4(fmaxf(h0.x, h1.x), fmaxf(h0.y, h1.y), fmaxf(h0.z, h1.z), 0.0f);
    const uint32_t c = a.cnt[i] + a.cnt[j];
    left[node] = a.ref[i];
    right[node] = a.ref[j];
    count[node] = c;
    blo[node] = lo;
    bhi[node] = hi;
    if (D.cost)   // the children's costs were written in earlier rounds
        dp_node(D, node, a.ref[i], half_area_box(xyz(l0), xyz(h0)), a.ref[j], half_area_box(xyz(l1), xyz(h1)), c,
                half_area_box(xyz(lo), xyz(hi)));
    b.ref[pos] = node;
    b.cnt[pos] = c;
    b.lo[pos] = lo;
    b.hi[pos] = hi;
}

// top-down layout of the nodes [lo, hi] (one round's merges; their parents are done): each
// node's range starts at first[node], its left subtree first; leaves take their position in
// perm and their child reference becomes LEAF_BIT | position
__global__ void k_ploc_layout(uint32_t lo, uint32_t hi, uint32_t* left, uint32_t* right, const uint32_t* count,
                              uint32_t* first, uint32_t* last, uint32_t* perm) {
    const uint32_t k = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (k > hi) return;
    const uint32_t f = first[k];
    const uint32_t L = left[k], R = right[k];
    const uint32_t cl = (L & LEAF_BIT) ? 1u : count[L];
    if (L & LEAF_BIT) {
        perm[f] = L & ~LEAF_BIT;
        left[k] = LEAF_BIT | f;
    } else {
        first[L] = f;
    }
    if (R & LEAF_BIT) {
        perm[f + cl] = R & ~LEAF_BIT;
        right[k] = LEAF_BIT | (f + cl);
    } else {
        first[R] = f + cl;
    }
    last[k] = f + count[k] - 1u;
}

// ------------------------------------------------------------------ collapse to wide nodes
struct CollapseCtx {
    BinTree T;
    uint32_t leaf_size;
    uint32_t width;         // most children of a wide node, 2..8
    uint32_t* task_ref;     // binary node ref of each wide-node task
    uint32_t* task_node;    // wide node index of each task
    uint32_t* counters;     // [0] node count, [1] triangle count, [2] queue tail
    uint4* nodes;
    float4* out_tris;
    const float4* in_tris;
    DpArrays dp;            // cost-optimal choices (dp.cost null: greedy, largest child first)
};

__device__ __forceinline__ uint32_t ref_count(const BinTree& T, uint32_t ref) {
    return (ref & LEAF_BIT) ? 1u : T.last[ref] - T.first[ref] + 1u;
}
__device__ __forceinline__ uint32_t ref_first(const BinTree& T, uint32_t ref) {
    return (ref & LEAF_BIT) ? (ref & ~LEAF_BIT) : T.first[ref];
}
__device__ __forceinline__ float area(const Box& b) {
    const float dx = b.hi.x - b.lo.x, dy = b.hi.y - b.lo.y, dz = b.hi.z - b.lo.z;
    return dx * dy + dy * dz + dz * dx;
}

__device__ __forceinline__ uint32_t pack_bytes(const uint32_t* q, int off) {
    return q[off] | (q[off + 1] << 8) | (q[off + 2] << 16) | (q[off + 3] << 24);
}

__global__ void k_collapse(CollapseCtx C, uint32_t qbeg, uint32_t qend) {
    const uint32_t ti = qbeg + blockIdx.x * blockDim.x + threadIdx.x;
    if (ti >= qend) return;
    const BinTree& T = C.T;
    const uint32_t root_ref = C.task_ref[ti];
    const uint32_t wnode = C.task_node[ti];
    uint32_t ch[8];
    Box cb[8];
    int nc = 0;
    if ((root_ref & LEAF_BIT) || ref_count(T, root_ref) <= C.leaf_size) {
        ch[0] = root_ref;
        cb[0] = ref_box(T, root_ref);
        nc = 1;
    } else if (C.dp.cost) {
        // unfold the choices: the root's split, then each part's split of its slot budget
        uint32_t sref[8], sj[8];
        int sp = 0;
        const uint32_t d0 = C.dp.dec[root_ref];
        const uint32_t j0 = min(max(d0 & 15u, 2u), 8u);
        const uint32_t i0 = (d0 >> (4u * (j0 - 1u))) & 15u;
        sref[sp] = T.right[root_ref]; sj[sp++] = j0 - i0;
        sref[sp] = T.left[root_ref]; sj[sp++] = i0;
        while (sp > 0) {
            const uint32_t r = sref[--sp], j = sj[sp];
            const uint32_t i = (r & LEAF_BIT) || j < 2u || j > 8u ? 0u : (C.dp.dec[r] >> (4u * (j - 1u))) & 15u;
            if (i == 0u || i >= j || nc + sp + 2 > 8) {   // one slot (valid choices never need the guards)
                ch[nc] = r;
                cb[nc] = ref_box(T, r);
                ++nc;
            } else {
                sref[sp] = T.right[r]; sj[sp++] = j - i;
                sref[sp] = T.left[r]; sj[sp++] = i;
            }
        }
    } else {
        ch[0] = T.left[root_ref];
        ch[1] = T.right[root_ref];
        cb[0] = ref_box(T, ch[0]);
        cb[1] = ref_box(T, ch[1]);
        nc = 2;
        while (nc < (int)C.width) {
            int best = -1;
            float best_a = -1.0f;
            for (int j = 0; j < nc; ++j) {
                if ((ch[j] & LEAF_BIT) || ref_count(T, ch[j]) <= C.leaf_size) continue;
                const float a = area(cb[j]);
                if (a > best_a) { best_a = a; best = j; }
            }
            if (best < 0) break;
            const uint32_t r = ch[best];
            ch[best] = T.left[r];
            cb[best] = ref_box(T, ch[best]);
            ch[nc] = T.right[r];
            cb[nc] = ref_box(T, ch[nc]);
            ++nc;
        }
    }
    uint32_t n_int = 0, n_leaf_tris = 0;
    for (int j = 0; j < nc; ++j) {
        const uint32_t c = ref_count(T, ch[j]);
        if (c > C.leaf_size) ++n_int; else n_leaf_tris += c;
    }
    const uint32_t child_base = n_int ? atomicAdd(&C.counters[0], n_int) : 0u;
    const uint32_t tri_base = n_leaf_tris ? atomicAdd(&C.counters[1], n_leaf_tris) : 0u;
    const uint32_t qpos = n_int ? atomicAdd(&C.counters[2], n_int) : 0u;
    // node box and quantisation frame
    Box nb = cb[0];
    for (int j = 1; j < nc; ++j) nb = box_union(nb, cb[j]);
    const float3 p = nb.lo;
    float ext[3] = {nb.hi.x - nb.lo.x, nb.hi.y - nb.lo.y, nb.hi.z - nb.lo.z};
    const float emax = fmaxf(ext[0], fmaxf(ext[1], ext[2]));
    uint32_t ebias[3];
    float scale[3];
    for (int a = 0; a < 3; ++a) {
        const float e = fmaxf(fmaxf(ext[a], emax * 1e-6f), 1e-30f);
        int ex;
        frexpf(e / 255.0f, &ex);
        int b = min(max(ex + 127, 1), 254);
        float sc = __uint_as_float((uint32_t)b << 23);
        while (b < 254 && fmaf(255.0f, sc, comp3(p, a)) < comp3(nb.hi, a)) { ++b; sc = __uint_as_float((uint32_t)b << 23); }
        ebias[a] = (uint32_t)b;
        scale[a] = sc;
    }
    uint32_t qlo[3][8], qhi[3][8], meta[8];
    uint32_t imask = 0, rank = 0, toff = 0;
    for (int j = 0; j < 8; ++j) {
        meta[j] = 0;
        for (int a = 0; a < 3; ++a) { qlo[a][j] = 0; qhi[a][j] = 0; }
    }
    for (int j = 0; j < nc; ++j) {
        for (int a = 0; a < 3; ++a) {
            const float pa = comp3(p, a), sc = scale[a];
            const float lo = comp3(cb[j].lo, a), hi = comp3(cb[j].hi, a);
            float ql = floorf(__fsub_rd(lo, pa) / sc);
            ql = fminf(fmaxf(ql, 0.0f), 255.0f);
            while (ql > 0.0f && fmaf(ql, sc, pa) > lo) ql -= 1.0f;
            float qh = ceilf(__fsub_ru(hi, pa) / sc);
            qh = fminf(fmaxf(qh, 0.0f), 255.0f);
            while (qh < 255.0f && fmaf(qh, sc, pa) < hi) qh += 1.0f;
            qlo[a][j] = (uint32_t)ql;
            qhi[a][j] = (uint32_t)qh;
        }
        const uint32_t c = ref_count(T, ch[j]);
        if (c > C.leaf_size) {
            imask |= 1u << j;
            meta[j] = 1u;
            C.task_ref[qpos + rank] = ch[j];
            C.task_node[qpos + rank] = child_base + rank;
            ++rank;
        } else {
            meta[j] = (c << 5) | toff;
            const uint32_t f = ref_first(T, ch[j]);
            for (uint32_t k = 0; k < c; ++k) {
                const uint32_t src = T.perm[f + k];
                const uint32_t dst = tri_base + toff + k;
                C.out_tris[3u * dst + 0] = C.in_tris[3u * src + 0];
                C.out_tris[3u * dst + 1] = C.in_tris[3u * src + 1];
                C.out_tris[3u * dst + 2] = C.in_tris[3u * src + 2];
            }
            toff += c;
        }
    }
    uint4* o = C.nodes + 5u * wnode;
    o[0] = make_uint4(__float_as_uint(p.x), __float_as_uint(p.y), __float_as_uint(p.z),
                      ebias[0] | (ebias[1] << 8) | (ebias[2] << 16) | (imask << 24));
    o[1] = make_uint4(child_base, tri_base, pack_bytes(meta, 0), pack_bytes(meta, 4));
    o[2] = make_uint4(pack_bytes(qlo[0], 0), pack_bytes(qlo[0], 4), pack_bytes(qlo[1], 0), pack_bytes(qlo[1], 4));
    o[3] = make_uint4(pack_bytes(qlo[2], 0), pack_bytes(qlo[2], 4), pack_bytes(qhi[0], 0), pack_bytes(qhi[0], 4));
    o[4] = make_uint4(pack_bytes(qhi[1], 0), pack_bytes(qhi[1], 4), pack_bytes(qhi[2], 0), pack_bytes(qhi[2], 4));
}

template <typename T>
static cudaError_t dalloc(T** p, size_t n) {
    return cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T));
}

pt_status pt_build_bvh_impl(pt_scene* s, uint32_t leaf_size, uint32_t builder, uint32_t collapse, float tri_cost,
                            float box_cost, uint32_t max_width, cudaStream_t st) {
    const uint32_t n = s->n_tris;
    if (s->d_nodes) { cudaFree(s->d_nodes); s->d_nodes = nullptr; }
    if (s->d_tris) { cudaFree(s->d_tris); s->d_tris = nullptr; }
    uint64_t *k0 = nullptr, *k1 = nullptr;
    uint32_t *v0 = nullptr, *v1 = nullptr, *hist = nullptr, *cb = nullptr;
    uint32_t *left = nullptr, *right = nullptr, *pint = nullptr, *pleaf = nullptr, *first = nullptr, *last = nullptr;
    uint32_t *flags = nullptr, *tref = nullptr, *tnode = nullptr, *counters = nullptr;
    float4 *blo = nullptr, *bhi = nullptr, *clo = nullptr, *chi = nullptr;
    float* dpc = nullptr;
    uint32_t* dpd = nullptr;
    const uint32_t nblocks = (n + RS_TILE - 1) / RS_TILE;
    pt_status status = PT_OK;
    auto cleanup = [&]() {
        void* ps[] = {k0,    k1,    v0,    v1,    hist,  cb,       left, right, pint, pleaf, first,
                      last,  flags, tref,  tnode, counters, blo,  bhi,   clo,  chi,  dpc,   dpd};
        for (void* q : ps)
            if (q) cudaFree(q);
    };
#define BTRY(call)                                                                           \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            pt_set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                \
            cleanup();                                                                       \
            return e_ == cudaErrorMemoryAllocation ? PT_ERR_OOM : PT_ERR_CUDA;               \
        }                                                                                    \
    } while (0)
    BTRY(dalloc(&k0, n)); BTRY(dalloc(&k1, n)); BTRY(dalloc(&v0, n)); BTRY(dalloc(&v1, n));
    BTRY(dalloc(&hist, (size_t)256 * nblocks)); BTRY(dalloc(&cb, 8));
    BTRY(dalloc(&left, n)); BTRY(dalloc(&right, n)); BTRY(dalloc(&pint, n)); BTRY(dalloc(&pleaf, n));
    BTRY(dalloc(&first, n)); BTRY(dalloc(&last, n)); BTRY(dalloc(&flags, n));
    BTRY(dalloc(&tref, n + 1)); BTRY(dalloc(&tnode, n + 1)); BTRY(dalloc(&counters, 4));
    BTRY(dalloc(&blo, n)); BTRY(dalloc(&bhi, n));
    if (builder == PT_BVH_PLOC) { BTRY(dalloc(&clo, (size_t)2 * n)); BTRY(dalloc(&chi, (size_t)2 * n)); }
    DpArrays D{nullptr, nullptr, leaf_size, tri_cost, box_cost, max_width};
    if (collapse == PT_COLLAPSE_OPTIMAL) {
        BTRY(dalloc(&dpc, (size_t)8 * n));
        BTRY(dalloc(&dpd, n));
        D.cost = dpc;
        D.dec = dpd;
    }
    BTRY(dalloc(&s->d_nodes, (size_t)5 * (n + 1)));
    BTRY(dalloc(&s->d_tris, (size_t)3 * n));

    const uint32_t cbinit[6] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u};
    BTRY(cudaMemcpyAsync(cb, cbinit, sizeof(cbinit), cudaMemcpyHostToDevice, st));
    const uint32_t g = (n + 255) / 256;
    PT_LAUNCH(k_centroid_bounds, g, 256, 0, st, s->d_tris_raw, n, cb);
    PT_LAUNCH(k_morton, g, 256, 0, st, s->d_tris_raw, n, cb, k0, v0);
    s->launches += 2;
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 8 * pass;
        PT_LAUNCH(k_rs_hist, nblocks, RS_THREADS, 0, st, k0, n, shift, hist, nblocks);
        PT_LAUNCH(k_rs_scan, 1, 1024, 0, st, hist, 256u * nblocks);
        PT_LAUNCH(k_rs_scatter, nblocks, RS_THREADS, 0, st, k0, v0, k1, v1, n, shift, hist, nblocks);
        std::swap(k0, k1);
        std::swap(v0, v1);
        s->launches += 3;
    }
    BinTree T;
    T.left = left; T.right = right; T.first = first; T.last = last; T.perm = v0;
    T.blo = blo; T.bhi = bhi; T.tris = s->d_tris_raw;
    if (n > 1 && builder == PT_BVH_LBVH) {
        PT_LAUNCH(k_karras, (n - 1 + 255) / 256, 256, 0, st, k0, (int)n, left, right, pint, pleaf, first, last);
        BTRY(cudaMemsetAsync(flags, 0, (size_t)n * sizeof(uint32_t), st));
        PT_LAUNCH(k_bottom_up, g, 256, 0, st, T, (int)n, pint, pleaf, flags, D);
        s->launches += 2;
    } else if (n > 1) {
        // PLOC over the Morton order: cluster arrays ping-pong between (tref, flags, clo, chi)
        // and (tnode, last, clo + n, chi + n); scan prefixes in k1, block totals in hist,
        // nearest neighbours in pint, node triangle counts in pleaf, the final order in v1
        Clusters ca{tref, flags, clo, chi}, cb2{tnode, last, clo + n, chi + n};
        uint64_t* pre = k1;
        uint64_t* bsum = reinterpret_cast<uint64_t*>(hist);
        PT_LAUNCH(k_ploc_init, g, 256, 0, st, s->d_tris_raw, v0, n, ca);
        s->launches++;
        std::vector<std::pair<uint32_t, uint32_t>> rounds;
        uint32_t m = n, merged = 0;
        while (m > 1) {
            const uint32_t nb = (m + PLOC_SCAN_TILE - 1) / PLOC_SCAN_TILE;
            PT_LAUNCH(k_ploc_nn, (m + PLOC_THREADS - 1) / PLOC_THREADS, PLOC_THREADS, 0, st, ca, m, pint);
            PT_LAUNCH(k_ploc_scan, nb, PLOC_THREADS, 0, st, pint, m, pre, bsum);
            PT_LAUNCH(k_ploc_scan_top, 1, 1024, 0, st, bsum, nb);
            PT_LAUNCH(k_ploc_compact, (m + 255) / 256, 256, 0, st, ca, cb2, pint, m, pre, bsum, n, merged, left,
                      right, pleaf, blo, bhi, D);
            s->launches += 4;
            uint64_t total = 0;
            BTRY(cudaMemcpyAsync(&total, bsum + nb, sizeof(total), cudaMemcpyDeviceToHost, st));
            BTRY(cudaStreamSynchronize(st));
            const uint32_t merges = (uint32_t)(total >> 32), m_new = (uint32_t)(total & 0xffffffffull);
            if (merges == 0 || m_new != m - merges || merged + merges > n - 1) {
                pt_set_error("PLOC clustering made no progress");
                cleanup();
                return PT_ERR_CUDA;
            }
            rounds.emplace_back(n - 1 - merged - merges, n - 2 - merged);
            merged += merges;
            m = m_new;
            std::swap(ca, cb2);
        }
        BTRY(cudaMemsetAsync(first, 0, sizeof(uint32_t), st));
        for (size_t r = rounds.size(); r-- > 0;) {
            const uint32_t lo = rounds[r].first, hi = rounds[r].second;
            PT_LAUNCH(k_ploc_layout, (hi - lo + 1 + 255) / 256, 256, 0, st, lo, hi, left, right, pleaf, first, last, v1);
            s->launches++;
        }
        T.perm = v1;
    }
    // collapse, one level per launch
    const uint32_t root_ref = n > 1 ? 0u : LEAF_BIT;
    const uint32_t init[4] = {1u, 0u, 1u, 0u};
    BTRY(cudaMemcpyAsync(counters, init, sizeof(init), cudaMemcpyHostToDevice, st));
    const uint32_t zero = 0;
    BTRY(cudaMemcpyAsync(tref, &root_ref, sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    BTRY(cudaMemcpyAsync(tnode, &zero, sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    CollapseCtx C;
    C.T = T;
    C.leaf_size = leaf_size;
    C.width = max_width;
    C.task_ref = tref;
    C.task_node = tnode;
    C.counters = counters;
    C.nodes = s->d_nodes;
    C.out_tris = s->d_tris;
    C.in_tris = s->d_tris_raw;
    C.dp = D;
    uint32_t qbeg = 0, qend = 1, depth = 0;
    uint32_t host_counters[4] = {0, 0, 0, 0};
    while (qbeg < qend) {
        const uint32_t cnt = qend - qbeg;
        PT_LAUNCH(k_collapse, (cnt + 127) / 128, 128, 0, st, C, qbeg, qend);
        s->launches++;
        BTRY(cudaMemcpyAsync(host_counters, counters, sizeof(host_counters), cudaMemcpyDeviceToHost, st));
        BTRY(cudaStreamSynchronize(st));
        ++depth;
        qbeg = qend;
        qend = host_counters[2];
        if (depth > 200) { pt_set_error("BVH collapse did not terminate"); status = PT_ERR_CUDA; break; }
    }
    BTRY(cudaGetLastError());
    if (status == PT_OK && host_counters[1] != n) {
        pt_set_error("BVH collapse placed " + std::to_string(host_counters[1]) + " of " + std::to_string(n) + " triangles");
        status = PT_ERR_CUDA;
    }
    s->n_nodes = host_counters[0];
    s->depth = depth;
    cleanup();
#undef BTRY
    return status;
}

// ------------------------------------------------------------------ environment tables
// weights w = luminance * sin(theta at the texel centre); per-row conditional CDF and the
// marginal CDF over rows; a row (or the whole map) of zero weight gets a uniform CDF.
__global__ void k_env_rows(const float* env, int w, int h, float* wtex, float* cond, float* rowsum) {
    __shared__ float part[256];
    __shared__ float running;
    const int y = blockIdx.x;
    const float st = sinf(PT_PI_F * ((float)y + 0.5f) / (float)h);
    if (threadIdx.x == 0) running = 0.0f;
    __syncthreads();
    float* cd = cond + (size_t)y * (w + 1);
    for (int base = 0; base < w; base += 256) {
        const int x = base + threadIdx.x;
        float wt = 0.0f;
        if (x < w) {
            const float* t = env + 3 * ((size_t)y * w + x);
            wt = fmaxf(lum3(mk3(t[0], t[1], t[2])) * st, 0.0f);
            wtex[(size_t)y * w + x] = wt;
        }
        part[threadIdx.x] = wt;
        __syncthreads();
        for (int off = 1; off < 256; off <<= 1) {
            const float v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0.0f;
            __syncthreads();
            part[threadIdx.x] += v;
            __syncthreads();
        }
        if (x < w) cd[x + 1] = running + part[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) running += part[255];
        __syncthreads();
    }
    const float tot = running;
    for (int x = threadIdx.x; x < w; x += 256) cd[x + 1] = tot > 0.0f ? cd[x + 1] / tot : (float)(x + 1) / (float)w;
    if (threadIdx.x == 0) {
        cd[0] = 0.0f;
        rowsum[y] = tot;
    }
}

__global__ void k_env_marg(const float* rowsum, int h, float* marg, float* total) {
    __shared__ float part[1024];
    __shared__ float running;
    if (threadIdx.x == 0) running = 0.0f;
    __syncthreads();
    for (int base = 0; base < h; base += 1024) {
        const int y = base + threadIdx.x;
        part[threadIdx.x] = y < h ? rowsum[y] : 0.0f;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const float v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0.0f;
            __syncthreads();
            part[threadIdx.x] += v;
            __syncthreads();
        }
        if (y < h) marg[y + 1] = running + part[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) running += part[1023];
        __syncthreads();
    }
    const float tot = running;
    for (int y = threadIdx.x; y < h; y += 1024) marg[y + 1] = tot > 0.0f ? marg[y + 1] / tot : (float)(y + 1) / (float)h;
    if (threadIdx.x == 0) {
        marg[0] = 0.0f;
        total[0] = tot;
    }
}

// search guides: guide[g] = the CDF index for u = g / G (see cdf_find_guided)
__global__ void k_env_guides(const float* marg, const float* cond, int w, int h, int gm, int gc, int* guide) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t <= gm) {
        guide[t] = cdf_find(marg, h, (float)t / (float)gm);
        return;
    }
    const int r = t - (gm + 1);
    if (r >= h * (gc + 1)) return;
    const int y = r / (gc + 1), g = r % (gc + 1);
    guide[t] = cdf_find(cond + (size_t)y * (w + 1), w, (float)g / (float)gc);
}

pt_status pt_build_env_impl(pt_scene* s, cudaStream_t st) {
    if (!s->d_env || s->env_w <= 0) { s->env_total = 0.0f; return PT_OK; }
    const int w = s->env_w, h = s->env_h;
    float* rowsum = nullptr;
    if (!s->d_env_wtex) {
        PT_CUDA_TRY(cudaMalloc(&s->d_env_wtex, (size_t)w * h * sizeof(float)));
        PT_CUDA_TRY(cudaMalloc(&s->d_env_cond, (size_t)h * (w + 1) * sizeof(float)));
        PT_CUDA_TRY(cudaMalloc(&s->d_env_marg, (size_t)(h + 1) * sizeof(float)));
        PT_CUDA_TRY(cudaMalloc(&s->d_env_total, sizeof(float)));
        int gm = 1, gc = 1;
        while (gm < h) gm <<= 1;
        while (gc < w) gc <<= 1;
        s->env_gm = gm;
        s->env_gc = gc;
        PT_CUDA_TRY(cudaMalloc(&s->d_env_guide, ((size_t)gm + 1 + (size_t)h * (gc + 1)) * sizeof(int)));
    }
    PT_CUDA_TRY(cudaMalloc(&rowsum, (size_t)h * sizeof(float)));
    PT_LAUNCH(k_env_rows, h, 256, 0, st, s->d_env, w, h, s->d_env_wtex, s->d_env_cond, rowsum);
    PT_LAUNCH(k_env_marg, 1, 1024, 0, st, rowsum, h, s->d_env_marg, s->d_env_total);
    const int ng = s->env_gm + 1 + h * (s->env_gc + 1);
    PT_LAUNCH(k_env_guides, (ng + 255) / 256, 256, 0, st, s->d_env_marg, s->d_env_cond, w, h, s->env_gm, s->env_gc,
              s->d_env_guide);
    s->launches += 3;
    PT_CUDA_TRY(cudaMemcpyAsync(&s->env_total, s->d_env_total, sizeof(float), cudaMemcpyDeviceToHost, st));
    PT_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(rowsum);
    return PT_OK;
}
