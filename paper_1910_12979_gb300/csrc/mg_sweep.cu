// mg_sweep.cu -- pipelined one-launch red-black Gauss-Seidel sweep (cell-centred, 3-D).
//
// One full sweep (red, then black) of the variable-coefficient 7-point
// operator, reading xin and writing xout (ping-pong).  A CTA owns a 32 x TY
// column tile and marches through a chunk of z-planes.  Every operand of a
// plane -- xin with a 2-cell halo, b and the three face-coefficient planes over
// the tile plus a 1-cell ring -- is copied into a 5-slot shared-memory ring by
// cp.async two planes ahead of its use, so the HBM latency of plane k+2
// overlaps the arithmetic of plane k.  Per plane:
//   red on plane k over the tile + ring (old black neighbours from xin), then
//   black on plane k-1 over the tile (new red neighbours), write plane k-1.
// The ring's red values are recomputed by neighbouring CTAs; that redundancy is
// what lets one launch replace two dependent colour passes.  The row arithmetic
// (order of the six face terms, boundary handling, the diagonal) is the same as
// k_gsrb's, so the result equals two colour passes bit for bit.
//
// Requirements (checked by the launcher): nx % 32 == 0, ny % TY == 0, nz >= 2,
// z not periodic.
#include "mg_device.cuh"

namespace mgp {

constexpr int kPX = 32;       // tile width
constexpr int kPSlots = 5;    // ring depth (planes)

template <typename T, int TY>
struct PipeSlot {
    T X[TY + 4][kPX + 4];     // xin, 2-cell halo
    T Bb[TY + 2][kPX + 2];    // b over the tile + ring
    T FX[TY + 2][kPX + 3];    // x-faces of the tile + ring cells
    T FY[TY + 3][kPX + 2];    // y-faces
    T FZ[TY + 2][kPX + 2];    // low z-faces of the plane
    T IV[TY + 2][kPX + 2];    // 1/diagonal (FP64 levels only)
};

template <typename T, int TY>
struct PipeShared {
    PipeSlot<T, TY> slot[kPSlots];
    T rs[3][TY + 2][kPX + 2];  // new red values, planes k-2..k
};

__device__ __forceinline__ void cp_async_elem(void* smem, const void* gmem, bool valid, int bytes)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? bytes : 0;  // src-size 0: zero fill, nothing read
    if (bytes == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// global index along an axis of n cells for a tile-local position, wrapped
// when periodic; -1 when outside a non-periodic axis.  faces: n + 1 entries.
__device__ __forceinline__ int axis_pos(int g, int n, bool periodic, bool faces)
{
    const int hi = faces ? n : n - 1;
    if (g >= 0 && g <= hi) return g;
    if (!periodic) return -1;
    return g < 0 ? g + n : g - n;
}

template <typename T, int TY>
struct PipeArrays {  // per-array copy geometry: columns, rows, elements per thread
    static constexpr int NT = kPX * TY;
    static constexpr int NX = (TY + 4) * (kPX + 4);
    static constexpr int NB = (TY + 2) * (kPX + 2);
    static constexpr int NFX = (TY + 2) * (kPX + 3);
    static constexpr int NFY = (TY + 3) * (kPX + 2);
    static constexpr int PX = (NX + NT - 1) / NT, PB = (NB + NT - 1) / NT, PFX = (NFX + NT - 1) / NT,
                         PFY = (NFY + NT - 1) / NT;
};

template <typename T, int TY>
__global__ void __launch_bounds__(kPX * TY)
k_gsrb_pipe(CellLevel<T> L, const T* __restrict__ xin, T* __restrict__ xout, const T* __restrict__ b, int kz)
{
    using A = PipeArrays<T, TY>;
    constexpr int TX = kPX, NT = A::NT, RX = TX + 4, QX = TX + 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PipeShared<T, TY>& sh = *reinterpret_cast<PipeShared<T, TY>*>(smem_raw);

    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * kz, z1 = min(z0 + kz, nz);
    const int tid = threadIdx.y * TX + threadIdx.x;
    const bool px = L.bc.lo[0] == BCP, py = L.bc.lo[1] == BCP;
    const bool has_iv = L.invd != nullptr;
    const size_t plane = (size_t)nx * ny, fxplane = (size_t)(nx + 1) * ny, fyplane = (size_t)nx * (ny + 1);

    // plane-independent in-plane offsets (-1: outside the domain -> zero fill)
    int offX[A::PX], offB[A::PB], offFX[A::PFX], offFY[A::PFY];
#pragma unroll
    for (int e = 0; e < A::PX; ++e) {
        const int q = tid + e * NT, ly = q / RX, lx = q - ly * RX;
        const int gx = axis_pos(x0 - 2 + lx, nx, px, false), gy = axis_pos(y0 - 2 + ly, ny, py, false);
        offX[e] = (q < A::NX && gx >= 0 && gy >= 0) ? gy * nx + gx : -1;
    }
#pragma unroll
    for (int e = 0; e < A::PB; ++e) {
        const int q = tid + e * NT, ly = q / QX, lx = q - ly * QX;
        const int gx = axis_pos(x0 - 1 + lx, nx, px, false), gy = axis_pos(y0 - 1 + ly, ny, py, false);
        offB[e] = (q < A::NB && gx >= 0 && gy >= 0) ? gy * nx + gx : -1;
    }
#pragma unroll
    for (int e = 0; e < A::PFX; ++e) {
        const int q = tid + e * NT, ly = q / (QX + 1), lx = q - ly * (QX + 1);
        const int fx = axis_pos(x0 - 1 + lx, nx, px, true), gy = axis_pos(y0 - 1 + ly, ny, py, false);
        offFX[e] = (q < A::NFX && fx >= 0 && gy >= 0) ? gy * (nx + 1) + fx : -1;
    }
#pragma unroll
    for (int e = 0; e < A::PFY; ++e) {
        const int q = tid + e * NT, ly = q / QX, lx = q - ly * QX;
        const int gx = axis_pos(x0 - 1 + lx, nx, px, false), fy = axis_pos(y0 - 1 + ly, ny, py, true);
        offFY[e] = (q < A::NFY && gx >= 0 && fy >= 0) ? fy * nx + gx : -1;
    }

    // stage plane p (X, b, faces for p < nz; the low z-face plane for p <= nz)
    auto issue = [&](int p) {
        if (p >= 0 && p <= nz) {
            PipeSlot<T, TY>& S = sh.slot[p % kPSlots];
            const bool cellp = p < nz;
            T* X = &S.X[0][0];
            T* Bb = &S.Bb[0][0];
            T* FX = &S.FX[0][0];
            T* FY = &S.FY[0][0];
            T* FZ = &S.FZ[0][0];
            T* IV = &S.IV[0][0];
#pragma unroll
            for (int e = 0; e < A::PX; ++e) {
                const int q = tid + e * NT;
                if (q < A::NX) cp_async_elem(X + q, xin + (cellp ? p * plane : 0) + (offX[e] < 0 ? 0 : offX[e]),
                                             cellp && offX[e] >= 0, sizeof(T));
            }
#pragma unroll
            for (int e = 0; e < A::PB; ++e) {
                const int q = tid + e * NT;
                if (q < A::NB) {
                    const size_t o = (offB[e] < 0 ? 0 : offB[e]);
                    cp_async_elem(Bb + q, b + (cellp ? p * plane : 0) + o, cellp && offB[e] >= 0, sizeof(T));
                    cp_async_elem(FZ + q, L.bz + p * plane + o, offB[e] >= 0, sizeof(T));
                    if (has_iv)
                        cp_async_elem(IV + q, L.invd + (cellp ? p * plane : 0) + o, cellp && offB[e] >= 0, sizeof(T));
                }
            }
#pragma unroll
            for (int e = 0; e < A::PFX; ++e) {
                const int q = tid + e * NT;
                if (q < A::NFX)
                    cp_async_elem(FX + q, L.bx + (cellp ? p * fxplane : 0) + (offFX[e] < 0 ? 0 : offFX[e]),
                                  cellp && offFX[e] >= 0, sizeof(T));
            }
#pragma unroll
            for (int e = 0; e < A::PFY; ++e) {
                const int q = tid + e * NT;
                if (q < A::NFY)
                    cp_async_elem(FY + q, L.by + (cellp ? p * fyplane : 0) + (offFY[e] < 0 ? 0 : offFY[e]),
                                  cellp && offFY[e] >= 0, sizeof(T));
            }
        }
        cp_async_commit();
    };

    // The row of cell (gx, gy, k) at ring position (lx, ly) (R1 coordinates),
    // in k_gsrb's order: x low, x high, y low, y high, z low, z high.
    // Neighbour values come from V(dx, dy, dz).
    auto row = [&](const PipeSlot<T, TY>& Sk, const PipeSlot<T, TY>& Sk1, int gx, int gy, int k, int lx, int ly,
                   auto V, T& off, T& dg) {
        off = T(0);
        dg = T(0);
        const T bxl = Sk.FX[ly][lx], bxh = Sk.FX[ly][lx + 1];
        if (gx > 0 || L.bc.lo[0] == BCP) { off += bxl * V(-1, 0, 0); dg += bxl; }
        else if (L.bc.lo[0] == BCD) { dg += T(2) * bxl; }
        if (gx < nx - 1 || L.bc.hi[0] == BCP) { off += bxh * V(1, 0, 0); dg += bxh; }
        else if (L.bc.hi[0] == BCD) { dg += T(2) * bxh; }
        const T byl = Sk.FY[ly][lx], byh = Sk.FY[ly + 1][lx];
        if (gy > 0 || L.bc.lo[1] == BCP) { off += byl * V(0, -1, 0); dg += byl; }
        else if (L.bc.lo[1] == BCD) { dg += T(2) * byl; }
        if (gy < ny - 1 || L.bc.hi[1] == BCP) { off += byh * V(0, 1, 0); dg += byh; }
        else if (L.bc.hi[1] == BCD) { dg += T(2) * byh; }
        const T bzl = Sk.FZ[ly][lx], bzh = Sk1.FZ[ly][lx];
        if (k > 0) { off += bzl * V(0, 0, -1); dg += bzl; }
        else if (L.bc.lo[2] == BCD) { dg += T(2) * bzl; }
        if (k < nz - 1) { off += bzh * V(0, 0, 1); dg += bzh; }
        else if (L.bc.hi[2] == BCD) { dg += T(2) * bzh; }
    };

    auto red = [&](int k) {
        const PipeSlot<T, TY>& Sk = sh.slot[k % kPSlots];
        const PipeSlot<T, TY>& Sk1 = sh.slot[(k + 1) % kPSlots];
        const PipeSlot<T, TY>& Skm = sh.slot[(k + kPSlots - 1) % kPSlots];
#pragma unroll
        for (int e = 0; e < A::PB; ++e) {
            const int q = tid + e * NT;
            if (q >= A::NB) continue;
            const int ly = q / QX, lx = q - ly * QX;
            const int gx = axis_pos(x0 - 1 + lx, nx, px, false), gy = axis_pos(y0 - 1 + ly, ny, py, false);
            if (gx < 0 || gy < 0 || ((gx + gy + k) & 1) != 0) continue;
            auto V = [&](int dx, int dy, int dz) -> T {
                const PipeSlot<T, TY>& S = dz < 0 ? Skm : (dz > 0 ? Sk1 : Sk);
                return S.X[ly + 1 + dy][lx + 1 + dx];
            };
            T off, dg;
            row(Sk, Sk1, gx, gy, k, lx, ly, V, off, dg);
            const T inv = has_iv ? Sk.IV[ly][lx] : recip(dg);
            sh.rs[k % 3][ly][lx] = (off - Sk.Bb[ly][lx]) * inv;
        }
    };

    auto black = [&](int k) {
        const int lx = threadIdx.x + 1, ly = threadIdx.y + 1;
        const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y;
        const size_t id = (size_t)k * plane + (size_t)gy * nx + gx;
        T v;
        if (((gx + gy + k) & 1) == 0) {
            v = sh.rs[k % 3][ly][lx];
        } else {
            const PipeSlot<T, TY>& Sk = sh.slot[k % kPSlots];
            const PipeSlot<T, TY>& Sk1 = sh.slot[(k + 1) % kPSlots];
            auto V = [&](int dx, int dy, int dz) -> T { return sh.rs[(k + dz + 3) % 3][ly + dy][lx + dx]; };
            T off, dg;
            row(Sk, Sk1, gx, gy, k, lx, ly, V, off, dg);
            const T inv = has_iv ? Sk.IV[ly][lx] : recip(dg);
            v = (off - Sk.Bb[ly][lx]) * inv;
        }
        xout[id] = v;
    };

    const int kfirst = max(z0 - 1, 0), klast = min(z1, nz - 1);
    const int p0 = kfirst - 1;
    issue(p0);
    issue(p0 + 1);
    issue(p0 + 2);
    issue(p0 + 3);
    for (int k = kfirst; k <= klast; ++k) {
        cp_async_wait<1>();  // planes <= k + 1 have landed (k + 2 may be in flight)
        __syncthreads();
        red(k);
        __syncthreads();
        if (k - 1 >= z0 && k - 1 < z1) black(k - 1);
        issue(k + 3);
    }
    if (z1 == nz) {
        __syncthreads();
        black(nz - 1);
    }
    cp_async_wait<0>();
}

template <typename T>
bool cell_gsrb_fused_ok(int dim, const CellLevel<T>& L)
{
    return dim == 3 && L.nx % kPX == 0 && L.ny % 8 == 0 && L.nz >= 2 && L.bc.lo[2] != BCP;
}

template <typename T>
void cell_gsrb_sweep(int dim, const CellLevel<T>& L, const T* xin, T* xout, const T* b, cudaStream_t s)
{
    constexpr int TY = 8;
    const size_t smem = sizeof(PipeShared<T, TY>);
    static bool attr_set = false;  // one attribute call per instantiation
    if (!attr_set) {
        cudaFuncSetAttribute(k_gsrb_pipe<T, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = true;
    }
    // a chunk of z-planes per CTA: about 4 CTAs per SM over 152 SMs
    const long long tiles = (long long)(L.nx / kPX) * (L.ny / TY);
    int kz = (int)((tiles * L.nz + 152 * 4 - 1) / (152 * 4));
    kz = kz < 8 ? 8 : kz;
    dim3 grid(L.nx / kPX, L.ny / TY, (L.nz + kz - 1) / kz);
    MGP_LAUNCH(k_gsrb_pipe<T, TY><<<grid, dim3(kPX, TY), smem, s>>>(L, xin, xout, b, kz));
}

template bool cell_gsrb_fused_ok<float>(int, const CellLevel<float>&);
template bool cell_gsrb_fused_ok<double>(int, const CellLevel<double>&);
template void cell_gsrb_sweep<float>(int, const CellLevel<float>&, const float*, float*, const float*, cudaStream_t);
template void cell_gsrb_sweep<double>(int, const CellLevel<double>&, const double*, double*, const double*,
                                      cudaStream_t);

}  // namespace mgp
