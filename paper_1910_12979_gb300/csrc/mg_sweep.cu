// mg_sweep.cu -- pipelined one-launch red-black Gauss-Seidel sweep (cell-centred, 3-D).
//
// One full sweep (red, then black) of the variable-coefficient 7-point
// operator, reading xin and writing xout (ping-pong).  A CTA owns a 32 x 8
// column tile and marches through a chunk of z-planes.  Every operand of a
// plane -- xin with a 2-cell halo, b and the three face-coefficient planes over
// the tile plus a 1-cell ring -- is copied into a 5-slot shared-memory ring by
// cp.async two planes ahead of its use, so the HBM latency of plane k+2
// overlaps the arithmetic of plane k.  Per plane:
//   red on plane k over the tile + ring (old black neighbours from xin):
//       thread t < 170 owns one red cell of the 34 x 10 ring region;
//   black on plane k-1 over the tile (new red neighbours): thread t < 128 owns
//       one red/black pair of the tile, computes the black cell and stores the
//       pair with one 8-byte write.
// The ring's red values are recomputed by neighbouring CTAs; that redundancy is
// what lets one launch replace two dependent colour passes.  The row arithmetic
// (order of the six face terms, boundary handling, the diagonal) is that of
// k_gsrb, so the result equals two colour passes bit for bit.
//
// Every staged array starts at column x0 - 2 (even, so pairs of cells can be
// copied 8 bytes at a time, and pairs never straddle a periodic wrap because nx
// is even).  Requirements (checked by the launcher): nx % 32 == 0,
// ny % 8 == 0, nz >= 2, z not periodic.
#include "mg_device.cuh"

namespace mgp {

constexpr int kPX = 32;        // tile width
constexpr int kPY = 8;         // tile height
constexpr int kPSlots = 5;     // ring depth (planes)
constexpr int kPW = kPX + 4;   // staged row width: columns x0-2 .. x0+33
constexpr int kPT = kPX * kPY; // threads
constexpr int kRedCells = (kPX + 2) * (kPY + 2) / 2;  // red cells of the tile + ring: 170

template <typename T>
struct PipeSlot {
    T X[kPY + 4][kPW];   // xin, rows y0-2 .. y0+9
    T Bb[kPY + 2][kPW];  // b, rows y0-1 .. y0+8
    T FZ[kPY + 2][kPW];  // low z-faces of the plane
    T IV[kPY + 2][kPW];  // 1/diagonal (FP64 levels only)
    T FY[kPY + 3][kPW];  // y-faces, rows y0-1 .. y0+9
    T FX[kPY + 2][kPW];  // x-faces x0-2 .. x0+33 of rows y0-1 .. y0+8
};

template <typename T>
struct PipeShared {
    PipeSlot<T> slot[kPSlots];
    T rs[3][kPY + 2][kPW];  // new red values of planes k-2..k (columns as Bb)
};

__device__ __forceinline__ void cp_async(void* smem, const void* gmem, bool valid, int bytes)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? bytes : 0;  // src-size 0: zero fill, nothing read
    if (bytes == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
    else if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
    else asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// global position along an axis of n cells (faces: n + 1 entries) for a
// tile-relative position, wrapped when periodic; -1 outside a non-periodic axis
__device__ __forceinline__ int axis_pos(int g, int n, bool periodic, bool faces)
{
    const int hi = faces ? n : n - 1;
    if (g >= 0 && g <= hi) return g;
    if (!periodic) return -1;
    return g < 0 ? g + n : g - n;
}

// One staged array: each thread copies at most one element pair (or element)
// per plane; its in-plane source offset is fixed for the whole march.
struct CopyDesc {
    int dst;  // element index within the slot array, or -1: no copy by this thread
    int src;  // in-plane element offset, or -1: outside the domain (zero fill)
};

// FAST: x and y periodic, so every in-plane face term is present and every
// staged position is inside the domain; the boundary logic reduces to the two
// z tests, which are uniform per plane.
template <typename T, bool FAST>
__global__ void __launch_bounds__(kPT)
k_gsrb_pipe(CellLevel<T> L, const T* __restrict__ xin, T* __restrict__ xout, const T* __restrict__ b, int kz)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PipeShared<T>& sh = *reinterpret_cast<PipeShared<T>*>(smem_raw);

    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int x0 = blockIdx.x * kPX, y0 = blockIdx.y * kPY;
    const int z0 = blockIdx.z * kz, z1 = min(z0 + kz, nz);
    const int tid = threadIdx.x;
    const bool px = L.bc.lo[0] == BCP, py = L.bc.lo[1] == BCP;
    const bool has_iv = L.invd != nullptr;
    const size_t plane = (size_t)nx * ny, fxplane = (size_t)(nx + 1) * ny, fyplane = (size_t)nx * (ny + 1);

    // ---- copy descriptors (pairs for X, Bb, FZ, IV, FY; single elements for FX)
    constexpr int PAIRS = kPW / 2;  // 18 pairs per row
    auto pair_desc = [&](int rows, int row0, int idx, bool face_rows, int pitch) {
        CopyDesc d{-1, -1};
        if (idx < rows * PAIRS) {
            const int r = idx / PAIRS, c = 2 * (idx - r * PAIRS);
            d.dst = r * kPW + c;
            const int gx = axis_pos(x0 - 2 + c, nx, px, false), gy = axis_pos(row0 + r, ny, py, face_rows);
            d.src = (gx >= 0 && gy >= 0) ? gy * pitch + gx : -1;
        }
        return d;
    };
    const CopyDesc dX = pair_desc(kPY + 4, y0 - 2, tid, false, nx);
    const CopyDesc dB = pair_desc(kPY + 2, y0 - 1, tid, false, nx);
    const CopyDesc dY = pair_desc(kPY + 3, y0 - 1, tid, true, nx);
    CopyDesc dF[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int q = tid + e * kPT;
        dF[e] = CopyDesc{-1, -1};
        if (q < (kPY + 2) * kPW) {
            const int r = q / kPW, c = q - r * kPW;
            dF[e].dst = q;
            const int fx = axis_pos(x0 - 2 + c, nx, px, true), gy = axis_pos(y0 - 1 + r, ny, py, false);
            dF[e].src = (fx >= 0 && gy >= 0) ? gy * (nx + 1) + fx : -1;
        }
    }
    constexpr int PB = 2 * sizeof(T);  // bytes of one pair

    auto issue = [&](int p) {
        if (p >= 0 && p <= nz) {
            PipeSlot<T>& S = sh.slot[p % kPSlots];
            const bool cellp = p < nz;
            const T* xp = xin + (cellp ? p * plane : 0);
            const T* bp = b + (cellp ? p * plane : 0);
            const T* zp = L.bz + p * plane;
            const T* yp = L.by + (cellp ? p * fyplane : 0);
            const T* fp = L.bx + (cellp ? p * fxplane : 0);
            if (dX.dst >= 0) cp_async(&S.X[0][0] + dX.dst, xp + (dX.src < 0 ? 0 : dX.src), cellp && dX.src >= 0, PB);
            if (dB.dst >= 0) {
                const int o = dB.src < 0 ? 0 : dB.src;
                cp_async(&S.Bb[0][0] + dB.dst, bp + o, cellp && dB.src >= 0, PB);
                cp_async(&S.FZ[0][0] + dB.dst, zp + o, dB.src >= 0, PB);
                if (has_iv) cp_async(&S.IV[0][0] + dB.dst, L.invd + (cellp ? p * plane : 0) + o, cellp && dB.src >= 0, PB);
            }
            if (dY.dst >= 0) cp_async(&S.FY[0][0] + dY.dst, yp + (dY.src < 0 ? 0 : dY.src), cellp && dY.src >= 0, PB);
#pragma unroll
            for (int e = 0; e < 2; ++e)
                if (dF[e].dst >= 0)
                    cp_async(&S.FX[0][0] + dF[e].dst, fp + (dF[e].src < 0 ? 0 : dF[e].src), cellp && dF[e].src >= 0,
                             sizeof(T));
        }
        cp_async_commit();
    };

    // ---- the row arithmetic, in k_gsrb's order.  (cx, cy): the cell's column
    // in the staged arrays (x0-2 origin) and its row in the ring arrays
    // (y0-1 origin); V(dx, dy, dz) returns the neighbour value.
    auto row = [&](const PipeSlot<T>& Sk, const PipeSlot<T>& Sk1, int gx, int gy, int k, int cx, int cy, auto V,
                   T& off, T& dg) {
        off = T(0);
        dg = T(0);
        const T bxl = Sk.FX[cy][cx], bxh = Sk.FX[cy][cx + 1];
        if (gx > 0 || L.bc.lo[0] == BCP) { off = fmadd(bxl, V(-1, 0, 0), off); dg += bxl; }
        else if (L.bc.lo[0] == BCD) { dg += T(2) * bxl; }
        if (gx < nx - 1 || L.bc.hi[0] == BCP) { off = fmadd(bxh, V(1, 0, 0), off); dg += bxh; }
        else if (L.bc.hi[0] == BCD) { dg += T(2) * bxh; }
        const T byl = Sk.FY[cy][cx], byh = Sk.FY[cy + 1][cx];
        if (gy > 0 || L.bc.lo[1] == BCP) { off = fmadd(byl, V(0, -1, 0), off); dg += byl; }
        else if (L.bc.lo[1] == BCD) { dg += T(2) * byl; }
        if (gy < ny - 1 || L.bc.hi[1] == BCP) { off = fmadd(byh, V(0, 1, 0), off); dg += byh; }
        else if (L.bc.hi[1] == BCD) { dg += T(2) * byh; }
        const T bzl = Sk.FZ[cy][cx], bzh = Sk1.FZ[cy][cx];
        if (k > 0) { off = fmadd(bzl, V(0, 0, -1), off); dg += bzl; }
        else if (L.bc.lo[2] == BCD) { dg += T(2) * bzl; }
        if (k < nz - 1) { off = fmadd(bzh, V(0, 0, 1), off); dg += bzh; }
        else if (L.bc.hi[2] == BCD) { dg += T(2) * bzh; }
    };

    // ---- red cell of this thread (t < 170): ring row ry, pair index rix
    const bool red_thread = tid < kRedCells;
    const int ry = tid / (kPX / 2 + 1), rix = tid - ry * (kPX / 2 + 1);
    const int rgy = axis_pos(y0 - 1 + ry, ny, py, false);
    // ---- black pair of this thread (t < 128): tile row by, pair bp
    const bool black_thread = tid < kPT / 2;
    const int by = tid / (kPX / 2), bp = tid - by * (kPX / 2);

    // FAST-path per-thread offsets for both plane parities (index 0: (1+gy+k) even)
    // (plain scalars picked with a select: a runtime-indexed array would live in local memory)
    const int fr0 = ry * kPW + 2 * rix + 1;               // red cell in the ring arrays (cx = lx + 1)
    const int fb0 = (by + 1) * kPW + 2 * bp + 2;          // black cell in the ring arrays (cx = bx + 2)
    const int rpar0 = (1 + (y0 - 1 + ry)) & 1;            // red column parity at k = 0 (wrap keeps parity)
    const int bpar0 = (x0 + y0 + by + 1) & 1;             // black column parity at k = 0

    // FAST row: x low, x high, y low, y high, z low, z high (k_gsrb's order)
    auto row_fast = [&](const T* FXp, const T* FYp, const T* FZk, const T* FZk1, int o, int k, auto V, T& off,
                        T& dg) {
        const T bxl = FXp[o], bxh = FXp[o + 1], byl = FYp[o], byh = FYp[o + kPW];
        off = fmadd(bxl, V(-1, 0, 0), T(0));
        dg = bxl;
        off = fmadd(bxh, V(1, 0, 0), off);
        dg += bxh;
        off = fmadd(byl, V(0, -1, 0), off);
        dg += byl;
        off = fmadd(byh, V(0, 1, 0), off);
        dg += byh;
        const T bzl = FZk[o], bzh = FZk1[o];
        if (k > 0) { off = fmadd(bzl, V(0, 0, -1), off); dg += bzl; }
        else if (L.bc.lo[2] == BCD) { dg += T(2) * bzl; }
        if (k < nz - 1) { off = fmadd(bzh, V(0, 0, 1), off); dg += bzh; }
        else if (L.bc.hi[2] == BCD) { dg += T(2) * bzh; }
    };

    auto red_fast = [&](int k, int sk, int sk1, int skm) {
        if (!red_thread) return;
        const int o = fr0 + (rpar0 ^ (k & 1));                 // ring-array offset of the red cell
        const PipeSlot<T>& Sk = sh.slot[sk];
        const T* X0 = &Sk.X[0][0] + kPW;                   // X row of ring row 0
        const T* Xm = &sh.slot[skm].X[0][0] + kPW;
        const T* Xp = &sh.slot[sk1].X[0][0] + kPW;
        auto V = [&](int dx, int dy, int dz) -> T {
            const T* Xs = dz < 0 ? Xm : (dz > 0 ? Xp : X0);
            return Xs[o + dy * kPW + dx];
        };
        T off, dg;
        row_fast(&Sk.FX[0][0], &Sk.FY[0][0], &Sk.FZ[0][0], &sh.slot[sk1].FZ[0][0], o, k, V, off, dg);
        const T inv = has_iv ? (&Sk.IV[0][0])[o] : recip(dg);
        (&sh.rs[k % 3][0][0])[o] = (off - (&Sk.Bb[0][0])[o]) * inv;
    };

    auto black_fast = [&](int k, int sk, int sk1) {
        if (!black_thread) return;
        const int q = bpar0 ^ (k & 1);                     // 1: black cell is the pair's second
        const int o = fb0 + q;
        const PipeSlot<T>& Sk = sh.slot[sk];
        const T* R0 = &sh.rs[k % 3][0][0];
        const T* Rm = &sh.rs[(k + 2) % 3][0][0];
        const T* Rp = &sh.rs[(k + 1) % 3][0][0];
        auto V = [&](int dx, int dy, int dz) -> T {
            const T* Rs = dz < 0 ? Rm : (dz > 0 ? Rp : R0);
            return Rs[o + dy * kPW + dx];
        };
        T off, dg;
        row_fast(&Sk.FX[0][0], &Sk.FY[0][0], &Sk.FZ[0][0], &sh.slot[sk1].FZ[0][0], o, k, V, off, dg);
        const T inv = has_iv ? (&Sk.IV[0][0])[o] : recip(dg);
        const T vb = (off - (&Sk.Bb[0][0])[o]) * inv;
        const T vr = R0[q ? o - 1 : o + 1];
        T* dst = xout + (size_t)k * plane + (size_t)(y0 + by) * nx + (x0 + 2 * bp);
        if (q) { dst[0] = vr; dst[1] = vb; }
        else { dst[0] = vb; dst[1] = vr; }
    };

    auto red = [&](int k) {
        if (!red_thread || rgy < 0) return;
        const int lx = 2 * rix + ((1 + rgy + k) & 1);  // ring column 0..33 of a red cell
        const int gx = axis_pos(x0 - 1 + lx, nx, px, false);
        if (gx < 0) return;
        const PipeSlot<T>& Sk = sh.slot[k % kPSlots];
        const PipeSlot<T>& Sk1 = sh.slot[(k + 1) % kPSlots];
        const PipeSlot<T>& Skm = sh.slot[(k + kPSlots - 1) % kPSlots];
        const int cx = lx + 1, cy = ry;
        auto V = [&](int dx, int dy, int dz) -> T {
            const PipeSlot<T>& S = dz < 0 ? Skm : (dz > 0 ? Sk1 : Sk);
            return S.X[cy + 1 + dy][cx + dx];
        };
        T off, dg;
        row(Sk, Sk1, gx, rgy, k, cx, cy, V, off, dg);
        const T inv = has_iv ? Sk.IV[cy][cx] : recip(dg);
        sh.rs[k % 3][cy][cx] = (off - Sk.Bb[cy][cx]) * inv;
    };

    auto black = [&](int k) {
        if (!black_thread) return;
        const int gy = y0 + by, xa = x0 + 2 * bp;          // the pair's first cell
        const int bx = 2 * bp + ((xa + gy + k + 1) & 1);    // black cell, tile column
        const int gx = x0 + bx;
        const int cx = bx + 2, cy = by + 1;
        const PipeSlot<T>& Sk = sh.slot[k % kPSlots];
        const PipeSlot<T>& Sk1 = sh.slot[(k + 1) % kPSlots];
        const int r0 = k % 3, rm = (k + 2) % 3, rp = (k + 1) % 3;
        auto V = [&](int dx, int dy, int dz) -> T {
            const int r = dz < 0 ? rm : (dz > 0 ? rp : r0);
            return sh.rs[r][cy + dy][cx + dx];
        };
        T off, dg;
        row(Sk, Sk1, gx, gy, k, cx, cy, V, off, dg);
        const T inv = has_iv ? Sk.IV[cy][cx] : recip(dg);
        const T vb = (off - Sk.Bb[cy][cx]) * inv;
        const T vr = sh.rs[r0][cy][cx + (bx & 1 ? -1 : 1)];  // the pair's red cell
        const size_t id = (size_t)k * plane + (size_t)gy * nx + xa;
        T* dst = xout + id;
        if (bx & 1) { dst[0] = vr; dst[1] = vb; }
        else { dst[0] = vb; dst[1] = vr; }
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
        const int sk = k % kPSlots, sk1 = (k + 1) % kPSlots, skm = (k + kPSlots - 1) % kPSlots;
        if (FAST) red_fast(k, sk, sk1, skm);
        else red(k);
        __syncthreads();
        if (k - 1 >= z0 && k - 1 < z1) {
            if (FAST) black_fast(k - 1, skm, sk);
            else black(k - 1);
        }
        issue(k + 3);
    }
    if (z1 == nz) {
        __syncthreads();
        if (FAST) black_fast(nz - 1, (nz - 1) % kPSlots, nz % kPSlots);
        else black(nz - 1);
    }
    cp_async_wait<0>();
}

template <typename T>
bool cell_gsrb_fused_ok(int dim, const CellLevel<T>& L)
{
    return dim == 3 && L.nx % kPX == 0 && L.ny % kPY == 0 && L.nz >= 2 && L.bc.lo[2] != BCP;
}

template <typename T>
void cell_gsrb_sweep(int dim, const CellLevel<T>& L, const T* xin, T* xout, const T* b, cudaStream_t s)
{
    const size_t smem = sizeof(PipeShared<T>);
    static bool attr_set = false;  // one attribute call per instantiation
    if (!attr_set) {
        cudaFuncSetAttribute(k_gsrb_pipe<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_gsrb_pipe<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = true;
    }
    const bool fast = L.bc.lo[0] == BCP && L.bc.lo[1] == BCP;
    // a chunk of z-planes per CTA: about 4 CTAs per SM over 152 SMs
    const long long tiles = (long long)(L.nx / kPX) * (L.ny / kPY);
    int kz = (int)((tiles * L.nz + 152 * 4 - 1) / (152 * 4));
    kz = kz < 8 ? 8 : kz;
    dim3 grid(L.nx / kPX, L.ny / kPY, (L.nz + kz - 1) / kz);
    if (fast) MGP_LAUNCH(k_gsrb_pipe<T, true><<<grid, kPT, smem, s>>>(L, xin, xout, b, kz));
    else MGP_LAUNCH(k_gsrb_pipe<T, false><<<grid, kPT, smem, s>>>(L, xin, xout, b, kz));
}

template bool cell_gsrb_fused_ok<float>(int, const CellLevel<float>&);
template bool cell_gsrb_fused_ok<double>(int, const CellLevel<double>&);
template void cell_gsrb_sweep<float>(int, const CellLevel<float>&, const float*, float*, const float*, cudaStream_t);
template void cell_gsrb_sweep<double>(int, const CellLevel<double>&, const double*, double*, const double*,
                                      cudaStream_t);

}  // namespace mgp
