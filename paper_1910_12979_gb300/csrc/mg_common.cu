// mg_common.cu -- reductions, vector helpers and the dense coarsest-level solve.
#include <atomic>

#include "mg_device.cuh"

namespace mgp {

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// Sum the kRedBlocks partials of slot q in a fixed order (kThreads threads):
// out = the sum (times *mul when mul is given), written by thread 0.
__device__ __forceinline__ void finalize_slot(const double* __restrict__ partials, int q, double* __restrict__ out,
                                              const double* __restrict__ mul, double* sh)
{
    double s = 0.0;
    for (int b = threadIdx.x; b < kRedBlocks; b += blockDim.x) s += partials[q * kRedBlocks + b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = mul ? sh[0] * *mul : sh[0];
    __syncthreads();
}

// Sum the kRedBlocks partials of each slot in a fixed order: out[q].
__global__ void k_finalize(const double* __restrict__ partials, int nslots, double* __restrict__ out,
                           const double* __restrict__ mul)
{
    __shared__ double sh[kThreads];
    for (int q = 0; q < nslots; ++q) finalize_slot(partials, q, out, mul, sh);
}

// One block per solve of a batch: slot 0 of its partials, as k_finalize.
__global__ void k_finalize_batch(const FinalItem* __restrict__ items, const int* __restrict__ run)
{
    __shared__ double sh[kThreads];
    const FinalItem& it = items[blockIdx.x];
    if (!run[it.solve]) return;
    finalize_slot(it.partials, 0, it.out, it.mul, sh);
}

void reduce_finalize_batch(const FinalItem* items, int count, const int* run, cudaStream_t s)
{
    MGP_LAUNCH(k_finalize_batch<<<count, kThreads, 0, s>>>(items, run));
}

void reduce_finalize(const double* partials, int nslots, double* out, cudaStream_t s, const double* mul)
{
    MGP_LAUNCH(k_finalize<<<1, kThreads, 0, s>>>(partials, nslots, out, mul));
}

__global__ void k_sum_sq(const double* __restrict__ v, size_t n, double* __restrict__ partials)
{
    double acc[2] = {0.0, 0.0};
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const double x = v[t];
        acc[0] += x;
        acc[1] += x * x;
    }
    block_reduce_store<2>(acc, partials);
}

void vec_sum_sq(const double* v, size_t n, double* partials, cudaStream_t s)
{
    MGP_LAUNCH(k_sum_sq<<<kRedBlocks, kThreads, 0, s>>>(v, n, partials));
}

__global__ void k_sub_mean(double* __restrict__ v, size_t n, const double* __restrict__ sum, double count)
{
    const double m = *sum / count;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        v[t] -= m;
}

void vec_sub_mean(double* v, size_t n, const double* sum, double count, cudaStream_t s)
{
    MGP_LAUNCH(k_sub_mean<<<kRedBlocks, kThreads, 0, s>>>(v, n, sum, count));
}

__global__ void k_copy64(double* __restrict__ d, const double* __restrict__ a, size_t n)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        d[t] = a[t];
}
// V: four elements per step with 16-byte accesses (all pointers 16-byte aligned), then the tail
template <bool V>
__global__ void k_to32(float* __restrict__ d, const double* __restrict__ a, size_t n)
{
    const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, st = (size_t)gridDim.x * blockDim.x;
    size_t done = 0;
    if (V) {
        const size_t n4 = n / 4;
        for (size_t t = t0; t < n4; t += st) {
            const double2 p = reinterpret_cast<const double2*>(a)[2 * t];
            const double2 q = reinterpret_cast<const double2*>(a)[2 * t + 1];
            reinterpret_cast<float4*>(d)[t] =
                make_float4(f64_to_f32_rn(p.x), f64_to_f32_rn(p.y), f64_to_f32_rn(q.x), f64_to_f32_rn(q.y));
        }
        done = 4 * n4;
    }
    for (size_t t = done + t0; t < n; t += st) d[t] = f64_to_f32_rn(a[t]);
}
template <bool V>
__global__ void k_axpy32(double* __restrict__ phi, const float* __restrict__ e, const double* __restrict__ scale,
                         size_t n)
{
    const double s = *scale;
    const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, st = (size_t)gridDim.x * blockDim.x;
    size_t done = 0;
    if (V) {
        const size_t n4 = n / 4;
        for (size_t t = t0; t < n4; t += st) {
            const float4 ev = reinterpret_cast<const float4*>(e)[t];
            double2* pp = reinterpret_cast<double2*>(phi) + 2 * t;
            double2 p = pp[0], q = pp[1];
            p.x = fmadd(s, f32_to_f64(ev.x), p.x);
            p.y = fmadd(s, f32_to_f64(ev.y), p.y);
            q.x = fmadd(s, f32_to_f64(ev.z), q.x);
            q.y = fmadd(s, f32_to_f64(ev.w), q.y);
            pp[0] = p;
            pp[1] = q;
        }
        done = 4 * n4;
    }
    for (size_t t = done + t0; t < n; t += st) phi[t] = fmadd(s, f32_to_f64(e[t]), phi[t]);
}
static inline bool al16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// Batched refinement updates: resident blocks walk the tiles of every solve
// whose run flag is set; each thread updates four entries as k_axpy32 does
// (the update is entrywise, so the partition changes nothing).
__global__ void __launch_bounds__(kThreads)
k_axpy32_batch(const AxpyItem* __restrict__ items, int count, int tiles, const int* __restrict__ run)
{
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (items[mid].tile0 <= tile) lo = mid;
            else hi = mid - 1;
        }
        const AxpyItem& it = items[lo];
        if (!run[it.solve]) continue;
        const int t = (tile - it.tile0) * kThreads + threadIdx.x;
        if (t >= it.n4) continue;
        const double s = *it.scale;
        const float4 ev = reinterpret_cast<const float4*>(it.e)[t];
        double2* pp = reinterpret_cast<double2*>(it.phi) + 2 * t;
        double2 p = pp[0], q = pp[1];
        p.x = fmadd(s, f32_to_f64(ev.x), p.x);
        p.y = fmadd(s, f32_to_f64(ev.y), p.y);
        q.x = fmadd(s, f32_to_f64(ev.z), q.x);
        q.y = fmadd(s, f32_to_f64(ev.w), q.y);
        pp[0] = p;
        pp[1] = q;
    }
}

int axpy_batch_grid(int tiles)
{
    static std::atomic<int> per{0};
    int p = per.load(std::memory_order_acquire);
    if (p == 0) {
        int dev = 0, sms = 0, b = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_axpy32_batch, kThreads, 0) != cudaSuccess || b < 1) b = 1;
        p = (sms > 0 ? sms : kNumSMs) * b;
        per.store(p, std::memory_order_release);
    }
    return tiles < p ? tiles : p;
}

void axpy_f32_batch(const AxpyItem* items, int count, int tiles, const int* run, int grid, cudaStream_t s)
{
    MGP_LAUNCH(k_axpy32_batch<<<grid, kThreads, 0, s>>>(items, count, tiles, run));
}

__global__ void k_to64(double* __restrict__ d, const float* __restrict__ a, size_t n)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        d[t] = f32_to_f64(a[t]);
}

// Residual of a zero initial guess: r = f, so the FP32 copy r / scale and its
// squared norm need no operator application.  Same traversal, grid and
// accumulation order as the cell FP64 residual kernel, whose result it equals
// bit for bit when x = 0.
__global__ void k_init_zero_guess(const double* __restrict__ f, float* __restrict__ r32,
                                  const double* __restrict__ scale, double* __restrict__ partials, int n)
{
    const int sh = pow2_shift(*scale);
    float acc = 0.f;
    const int nquad = (n + 3) / 4;   // quads of consecutive entries, as the cell FP64 residual kernels
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nquad; u += gridDim.x * blockDim.x)
        for (int t = 4 * u; t < 4 * u + 4 && t < n; ++t) {
            const float rs = f64_to_f32_pow2(f[t], sh);
            acc = fmaf(rs, rs, acc);
            if (r32) r32[t] = rs;
        }
    double a[1] = {(double)acc};
    block_reduce_store<1>(a, partials);
}

void vec_init_zero_guess(const double* f, float* r32, const double* scale, double* partials, size_t n,
                         cudaStream_t s)
{
    MGP_LAUNCH(k_init_zero_guess<<<kRedBlocks, kThreads, 0, s>>>(f, r32, scale, partials, (int)n));
}

__global__ void k_recip(double* __restrict__ d, const double* __restrict__ a, size_t n)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        d[t] = recip_nr(a[t]);
}

void vec_recip(double* dst, const double* src, size_t n, cudaStream_t s)
{
    MGP_LAUNCH(k_recip<<<kRedBlocks, kThreads, 0, s>>>(dst, src, n));
}

void vec_to_f64(double* dst, const float* src, size_t n, cudaStream_t s)
{
    MGP_LAUNCH(k_to64<<<kRedBlocks, kThreads, 0, s>>>(dst, src, n));
}

void vec_copy_f64(double* dst, const double* src, size_t n, cudaStream_t s)
{
    MGP_LAUNCH(k_copy64<<<kRedBlocks, kThreads, 0, s>>>(dst, src, n));
}
__global__ void k_to32_pow2(float* __restrict__ d, const double* __restrict__ a, size_t n, int sh)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        d[t] = f64_to_f32_pow2(a[t], sh);
}
void vec_to_f32_pow2(float* dst, const double* src, size_t n, int shift, cudaStream_t s)
{
    MGP_LAUNCH(k_to32_pow2<<<kRedBlocks, kThreads, 0, s>>>(dst, src, n, shift));
}

void vec_to_f32(float* dst, const double* src, size_t n, cudaStream_t s)
{
    if (al16(dst) && al16(src)) MGP_LAUNCH(k_to32<true><<<kRedBlocks, kThreads, 0, s>>>(dst, src, n));
    else MGP_LAUNCH(k_to32<false><<<kRedBlocks, kThreads, 0, s>>>(dst, src, n));
}
void vec_zero_f32(float* v, size_t n, cudaStream_t s) { cudaMemsetAsync(v, 0, n * sizeof(float), s); }
void vec_zero_f64(double* v, size_t n, cudaStream_t s) { cudaMemsetAsync(v, 0, n * sizeof(double), s); }
void vec_axpy_f32(double* phi, const float* e, const double* scale, size_t n, cudaStream_t s)
{
    if (al16(phi) && al16(e)) MGP_LAUNCH(k_axpy32<true><<<kRedBlocks, kThreads, 0, s>>>(phi, e, scale, n));
    else MGP_LAUNCH(k_axpy32<false><<<kRedBlocks, kThreads, 0, s>>>(phi, e, scale, n));
}

__global__ void k_fscale(DevScalars* d) { set_fscale(d); }
void scalars_set_fscale(DevScalars* d, cudaStream_t s) { MGP_LAUNCH(k_fscale<<<1, 1, 0, s>>>(d)); }

// ------------------------------------------------------------ dense solve
//
// Gauss-Jordan with partial pivoting on [A | I] held in global memory, one CTA.
// A: n x n (n = N + 1 when the problem is singular: the bordered matrix
// [A 1; 1^T 0], whose inverse's leading N x N block maps a compatible b to the
// zero-mean solution).  Minv receives the leading N x N block, row-major.
constexpr int kGJThreads = 1024;

__global__ void k_border(double* A, int N, int lda)
{
    for (int t = threadIdx.x; t <= N; t += blockDim.x) {
        A[(size_t)t * lda + N] = t < N ? 1.0 : 0.0;
        A[(size_t)N * lda + t] = t < N ? 1.0 : 0.0;
    }
}

__global__ void __launch_bounds__(kGJThreads) k_gauss_jordan(double* __restrict__ W, int n, int* __restrict__ info)
{
    // W: n rows x 2n columns, row-major; left half A, right half I (set here)
    const int ld = 2 * n;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int r = t / n, c = t % n;
        W[(size_t)r * ld + n + c] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    __shared__ double sv[kGJThreads / 32];
    __shared__ int si[kGJThreads / 32];
    __shared__ int piv;
    __shared__ double pval;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) *info = 0;
    for (int k = 0; k < n; ++k) {
        // pivot search over rows k..n-1 (ties -> smallest row: deterministic)
        double best = -1.0;
        int bi = n;
        for (int r = k + threadIdx.x; r < n; r += blockDim.x) {
            const double v = fabs(W[(size_t)r * ld + k]);
            if (v > best || (v == best && r < bi)) { best = v; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { sv[warp] = best; si[warp] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = -1.0;
            int p = n;
            for (int w = 0; w < kGJThreads / 32; ++w)
                if (sv[w] > b || (sv[w] == b && si[w] < p)) { b = sv[w]; p = si[w]; }
            piv = p;
            pval = (p < n) ? W[(size_t)p * ld + k] : 0.0;
            if (b <= 0.0 && *info == 0) *info = k + 1;
        }
        __syncthreads();
        if (pval == 0.0) return;  // singular: info set, Minv left unusable
        const int p = piv;
        if (p != k)
            for (int c = threadIdx.x; c < ld; c += blockDim.x) {
                const double tmp = W[(size_t)k * ld + c];
                W[(size_t)k * ld + c] = W[(size_t)p * ld + c];
                W[(size_t)p * ld + c] = tmp;
            }
        __syncthreads();
        const double inv = 1.0 / pval;
        for (int c = threadIdx.x; c < ld; c += blockDim.x) W[(size_t)k * ld + c] *= inv;
        __syncthreads();
        // eliminate column k from every other row
        for (int t = threadIdx.x; t < n * ld; t += blockDim.x) {
            const int r = t / ld, c = t % ld;
            if (r == k || c == k) continue;
            W[(size_t)r * ld + c] -= W[(size_t)r * ld + k] * W[(size_t)k * ld + c];
        }
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += blockDim.x)
            if (r != k) W[(size_t)r * ld + k] = 0.0;
        __syncthreads();
    }
}

// Same elimination with the augmented matrix resident in shared memory
// (n <= kGJSmemMax): one global read of A, one global write of Minv.  Per
// pivot column k: warp 0 finds the pivot (largest |entry|, smallest row on
// ties); then the pivot row is swapped in, scaled and kept in prow; then every
// other row is updated over the columns right of k only.  Columns left of k
// are never read again (the inverse is the right half), so they are neither
// updated nor cleared.  Three barriers per column.
constexpr int kGJSmemMax = 112;

__global__ void __launch_bounds__(kGJThreads) k_gauss_jordan_smem(const double* __restrict__ A, int n, int N,
                                                                 double* __restrict__ Minv, int* __restrict__ info)
{
    extern __shared__ double W[];  // n x 2n
    __shared__ double prow[2 * kGJSmemMax];
    __shared__ int piv;
    __shared__ double pval;
    const int ld = 2 * n;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    for (int t = tid; t < n * ld; t += nt) {
        const int r = t / ld, c = t - r * ld;
        W[t] = c < n ? A[(size_t)r * ld + c] : ((c - n) == r ? 1.0 : 0.0);
    }
    if (tid == 0) *info = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (warp == 0) {
            double b = -1.0;
            int p = k;
            for (int r = k + lane; r < n; r += 32) {
                const double v = fabs(W[r * ld + k]);
                if (v > b) { b = v; p = r; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, b, o);
                const int op = __shfl_xor_sync(0xffffffffu, p, o);
                if (ob > b || (ob == b && op < p)) { b = ob; p = op; }
            }
            if (lane == 0) {
                piv = p;
                pval = W[p * ld + k];
                if (b <= 0.0) *info = k + 1;
            }
        }
        __syncthreads();
        const double pv = pval;
        if (pv == 0.0) return;
        const int p = piv;
        const double inv = 1.0 / pv;
        for (int c = k + tid; c < ld; c += nt) {
            const double a = W[k * ld + c], b = W[p * ld + c];
            if (p != k) W[p * ld + c] = a;
            const double s = b * inv;
            W[k * ld + c] = s;
            prow[c] = s;
        }
        __syncthreads();
        const int wdt = ld - k - 1;  // columns k+1 .. ld-1
        int r = tid / wdt, c = tid - r * wdt;
        const int dr = nt / wdt, dc = nt - dr * wdt;
        for (; r < n;) {
            if (r != k) W[r * ld + k + 1 + c] -= W[r * ld + k] * prow[k + 1 + c];
            c += dc;
            r += dr;
            if (c >= wdt) { c -= wdt; ++r; }
        }
        __syncthreads();
    }
    for (int t = tid; t < N * N; t += nt) {
        const int r = t / N, c = t - r * N;
        Minv[t] = W[r * ld + n + c];
    }
}

__global__ void k_extract(const double* __restrict__ W, int n, int N, double* __restrict__ Minv)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N * N; t += gridDim.x * blockDim.x) {
        const int r = t / N, c = t % N;
        Minv[t] = W[(size_t)r * 2 * n + n + c];
    }
}

// A must be laid out with lda = 2 * n (n = N or N + 1); the caller assembled
// the leading N x N block.  Returns 0 on success (after a device sync).
int dense_invert(double* A, int N, int singular, double* Minv, int* info, cudaStream_t s)
{
    const int n = N + (singular ? 1 : 0);
    if (singular) MGP_LAUNCH(k_border<<<1, 256, 0, s>>>(A, N, 2 * n));
    if (n <= kGJSmemMax) {
        const size_t smem = (size_t)n * 2 * n * sizeof(double);
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_gauss_jordan_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kGJSmemMax * 2 * kGJSmemMax * sizeof(double)));
            attr = true;
        }
        MGP_LAUNCH(k_gauss_jordan_smem<<<1, kGJThreads, smem, s>>>(A, n, N, Minv, info));
        return 0;
    }
    MGP_LAUNCH(k_gauss_jordan<<<1, kGJThreads, 0, s>>>(A, n, info));
    MGP_LAUNCH(k_extract<<<64, 256, 0, s>>>(A, n, N, Minv));
    return 0;
}

// x = Minv b, one warp per row
template <typename T>
__global__ void k_dense_apply(const double* __restrict__ Minv, int N, const T* __restrict__ b, T* __restrict__ x)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = warp; r < N; r += nw) {
        const double s = dense_row(Minv, N, b, r, lane);
        if (lane == 0) x[r] = from_f64<T>(s);
    }
}

template <typename T>
void dense_apply(const double* Minv, int N, const T* b, T* x, cudaStream_t s)
{
    const int blocks = ceil_div((long long)N * 32, kThreads);
    MGP_LAUNCH(k_dense_apply<T><<<blocks < 64 ? blocks : 64, kThreads, 0, s>>>(Minv, N, b, x));
}

template void dense_apply<float>(const double*, int, const float*, float*, cudaStream_t);
template void dense_apply<double>(const double*, int, const double*, double*, cudaStream_t);

}  // namespace mgp
