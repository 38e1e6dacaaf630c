// Locality reordering of a CSR matrix: the rows ordered by their entry count, descending (ties by
// row index), and the symmetric permutation B = P A P^T that relabels rows and columns alike.
// A power-law graph's hubs then occupy the first rows, so the neighbour rows most entries gather
// stay together in L2. B's log-determinant equals A's, and with the probe rows generated by the
// original row index (k_probes' row map) the estimator sees the same probes in another row order:
// the estimate changes only by the order of its sums.
//
//   order:   per chunk of ORD_CHUNK rows a histogram of the entry counts (ORD_BUCKETS buckets, the
//            last one holding every longer row), bucket starts in descending order, then each
//            chunk scatters its rows in row order within each bucket (a warp ranks equal buckets
//            with __match_any_sync): perm[new] = old, inv[old] = new. Deterministic.
//   permute: new row i = old row perm[i]; its columns mapped by inv, in the old row's order; src[e']
//            = the old entry of new entry e' (the values are gathered through it at every call).
//   hash:    an order-independent checksum of (rowptr, colind), to tell a changed structure from
//            the cached one.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace ll {

namespace {

constexpr int ORD_THREADS = 256;
constexpr int ORD_BUCKETS = 1024;   // entry counts 0 .. 1022 exactly, 1023 and above together
constexpr int ORD_CHUNK = 8192;     // rows per histogram / scatter chunk

__device__ __forceinline__ int row_bucket(const int32_t* rowptr, int r) {
    const int d = rowptr[r + 1] - rowptr[r];
    return d < ORD_BUCKETS - 1 ? d : ORD_BUCKETS - 1;
}

// counts[c * ORD_BUCKETS + b]: rows of chunk c in bucket b
__global__ void k_order_hist(const int32_t* rowptr, int n, int* counts) {
    __shared__ int h[ORD_BUCKETS];
    for (int b = threadIdx.x; b < ORD_BUCKETS; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const int r0 = blockIdx.x * ORD_CHUNK, r1 = min(n, r0 + ORD_CHUNK);
    for (int r = r0 + (int)threadIdx.x; r < r1; r += blockDim.x) atomicAdd(&h[row_bucket(rowptr, r)], 1);
    __syncthreads();
    for (int b = threadIdx.x; b < ORD_BUCKETS; b += blockDim.x) counts[(size_t)blockIdx.x * ORD_BUCKETS + b] = h[b];
}

// offsets[c * ORD_BUCKETS + b]: first position of chunk c's rows of bucket b, buckets in descending
// order, chunks ascending within a bucket. One CTA: the bucket totals, their scan, the chunk scans.
__global__ void k_order_offsets(const int* counts, int nchunks, int* offsets) {
    __shared__ int tot[ORD_BUCKETS];
    __shared__ int start[ORD_BUCKETS];
    for (int b = threadIdx.x; b < ORD_BUCKETS; b += blockDim.x) {
        int t = 0;
        for (int c = 0; c < nchunks; ++c) t += counts[(size_t)c * ORD_BUCKETS + b];
        tot[b] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int b = ORD_BUCKETS - 1; b >= 0; --b) {
            start[b] = acc;
            acc += tot[b];
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < ORD_BUCKETS; b += blockDim.x) {
        int acc = start[b];
        for (int c = 0; c < nchunks; ++c) {
            offsets[(size_t)c * ORD_BUCKETS + b] = acc;
            acc += counts[(size_t)c * ORD_BUCKETS + b];
        }
    }
}

// one warp per chunk: rows in order, 32 at a time; lanes of equal bucket take consecutive
// positions in lane order
__global__ void k_order_scatter(const int32_t* rowptr, int n, const int* offsets, int32_t* perm, int32_t* inv) {
    __shared__ int pos[ORD_BUCKETS];
    for (int b = threadIdx.x; b < ORD_BUCKETS; b += blockDim.x) pos[b] = offsets[(size_t)blockIdx.x * ORD_BUCKETS + b];
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const unsigned lt = (1u << lane) - 1u;
    const int r0 = blockIdx.x * ORD_CHUNK, r1 = min(n, r0 + ORD_CHUNK);
    for (int g = r0; g < r1; g += 32) {
        const int r = g + lane;
        const bool ok = r < r1;
        const int b = ok ? row_bucket(rowptr, r) : -1 - lane;   // distinct keys for the idle lanes
        const unsigned m = __match_any_sync(0xffffffffu, b);
        const int base = ok ? pos[b] : 0;
        __syncwarp();
        if (ok) {
            const int p = base + __popc(m & lt);
            perm[p] = r;
            inv[r] = p;
            if ((m & lt) == 0) pos[b] = base + __popc(m);   // the group's first lane advances the bucket
        }
        __syncwarp();
    }
}

// newdeg[i] = entries of old row perm[i]
__global__ void k_perm_degrees(const int32_t* rowptr, const int32_t* perm, int n, int* newdeg) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int o = perm[i];
        newdeg[i] = rowptr[o + 1] - rowptr[o];
    }
}

// exclusive scan of x[0..n) into out[0..n] (out[n] = total), in blocks of ORD_SCAN elements: the
// block sums, their scan by one CTA, then each block's local scan plus its offset
constexpr int ORD_SCAN = 1024;
__global__ void k_scan_blocks(const int* x, int n, int* bsum) {
    __shared__ int s[ORD_THREADS];
    const int b0 = blockIdx.x * ORD_SCAN;
    int t = 0;
    for (int i = threadIdx.x; i < ORD_SCAN && b0 + i < n; i += blockDim.x) t += x[b0 + i];
    s[threadIdx.x] = t;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = s[0];
}
__global__ void k_scan_sums(int* bsum, int nb, int* total) {
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b < nb; ++b) {
            const int v = bsum[b];
            bsum[b] = acc;
            acc += v;
        }
        *total = acc;
    }
}
__global__ void k_scan_apply(const int* x, int n, const int* boff, int32_t* out) {
    __shared__ int s[ORD_SCAN];
    const int b0 = blockIdx.x * ORD_SCAN;
    for (int i = threadIdx.x; i < ORD_SCAN; i += blockDim.x) s[i] = b0 + i < n ? x[b0 + i] : 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = boff[blockIdx.x];
        for (int i = 0; i < ORD_SCAN; ++i) {
            const int v = s[i];
            s[i] = acc;
            acc += v;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ORD_SCAN && b0 + i < n; i += blockDim.x) out[b0 + i] = s[i];
}

// one warp per new row: its entries copied from the old row with the columns relabelled
__global__ void k_permute_csr(const int32_t* rowptr, const int32_t* colind, int n, const int32_t* perm,
                              const int32_t* inv, const int32_t* rowptr_new, int32_t* colind_new, int32_t* src) {
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += gridDim.x * wpb) {
        const int o = perm[i];
        const int a = rowptr[o], e = rowptr[o + 1], d = rowptr_new[i];
        for (int k = a + lane; k < e; k += 32) {
            colind_new[d + (k - a)] = inv[colind[k]];
            src[d + (k - a)] = k;
        }
    }
}

// order-independent checksum of the structure (64-bit sums of index-weighted mixes)
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}
__global__ void k_structure_hash(const int32_t* rowptr, const int32_t* colind, int n, int64_t nnz, unsigned long long* out) {
    unsigned long long acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz; i += stride)
        acc += mix64(((unsigned long long)i << 32) ^ (unsigned long long)(uint32_t)colind[i]);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += stride)
        acc += mix64(0x9e3779b97f4a7c15ull ^ ((unsigned long long)i << 32) ^ (unsigned long long)(uint32_t)rowptr[i]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

}  // namespace

size_t reorder_work_bytes(int n) {
    const size_t nchunks = ((size_t)n + ORD_CHUNK - 1) / ORD_CHUNK;
    const size_t nb = ((size_t)n + ORD_SCAN - 1) / ORD_SCAN;
    return (2 * nchunks * ORD_BUCKETS + (size_t)n + nb + 4) * sizeof(int);
}

cudaError_t launch_reorder(const int32_t* rowptr, const int32_t* colind, int n, int32_t* perm, int32_t* inv,
                           int32_t* rowptr_new, int32_t* colind_new, int32_t* src, void* work, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int nchunks = (n + ORD_CHUNK - 1) / ORD_CHUNK;
    const int nb = (n + ORD_SCAN - 1) / ORD_SCAN;
    int* counts = static_cast<int*>(work);
    int* offsets = counts + (size_t)nchunks * ORD_BUCKETS;
    int* newdeg = offsets + (size_t)nchunks * ORD_BUCKETS;
    int* bsum = newdeg + n;
    int* total = bsum + nb;
    k_order_hist<<<nchunks, ORD_THREADS, 0, s>>>(rowptr, n, counts);
    k_order_offsets<<<1, 1024, 0, s>>>(counts, nchunks, offsets);
    k_order_scatter<<<nchunks, 256, 0, s>>>(rowptr, n, offsets, perm, inv);
    const int g = std::min(152 * 16, (n + ORD_THREADS - 1) / ORD_THREADS);
    k_perm_degrees<<<g, ORD_THREADS, 0, s>>>(rowptr, perm, n, newdeg);
    k_scan_blocks<<<nb, ORD_THREADS, 0, s>>>(newdeg, n, bsum);
    k_scan_sums<<<1, 32, 0, s>>>(bsum, nb, total);
    k_scan_apply<<<nb, ORD_THREADS, 0, s>>>(newdeg, n, bsum, rowptr_new);
    cudaError_t e = cudaMemcpyAsync(rowptr_new + n, total, sizeof(int), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    k_permute_csr<<<std::min(152 * 16, (n + 7) / 8), 256, 0, s>>>(rowptr, colind, n, perm, inv, rowptr_new, colind_new, src);
    return cudaGetLastError();
}

cudaError_t launch_structure_hash(const int32_t* rowptr, const int32_t* colind, int n, int64_t nnz,
                                  unsigned long long* out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_structure_hash<<<152 * 8, 256, 0, s>>>(rowptr, colind, n, nnz, out);
    return cudaGetLastError();
}

}  // namespace ll
