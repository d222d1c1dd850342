// Largest connected component, mass / spring topology and initial state: one thread block per
// robot.  Integer work is deterministic and matches the definition exactly:
//   * components are 6-connected sets of occupied voxels; the kept one is the largest, ties
//     broken toward the component holding the smallest linear voxel index;
//   * masses are the corners of kept voxels in ascending corner id;
//   * springs are the distinct corner pairs of kept voxels, sorted by (a, b), with stiffness and
//     actuation terms averaged over the kept voxels sharing the pair (Section II-A, Table II).
#include <cfloat>
#include <climits>

#include "common.cuh"

namespace vx {
namespace {

constexpr int kTopoThreads = 1024;

// The 13 corner offsets (dx, dy, dz) that point to a larger corner id, in increasing order of
// (dz, dy, dx): from a fixed corner they reach larger corners in increasing corner-id order.
// The step kernels use the same numbering (lattice_dir in common.cuh).
__constant__ int8_t c_dir[13][3] = {
    {1, 0, 0},   {-1, 1, 0}, {0, 1, 0},  {1, 1, 0},  {-1, -1, 1}, {0, -1, 1}, {1, -1, 1},
    {-1, 0, 1},  {0, 0, 1},  {1, 0, 1},  {-1, 1, 1}, {0, 1, 1},   {1, 1, 1}};

__device__ __forceinline__ int block_exclusive_scan(int val, int* sh, int* total)
{
    // Work-efficient enough for 1024 threads: warp scan + scan of warp totals.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = val;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int nw = (blockDim.x + 31) >> 5;
        int t = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) sh[lane] = t;   // inclusive warp totals
    }
    __syncthreads();
    int base = warp > 0 ? sh[warp - 1] : 0;
    int nw = (blockDim.x + 31) >> 5;
    if (total) *total = sh[nw - 1];
    __syncthreads();
    return base + x - val;
}

// Spring between corner (ci, cj, ck) and its neighbour along direction d: number of kept voxels
// containing both corners and the sums of their parameters.
__device__ __forceinline__ int spring_incidence(int ci, int cj, int ck, int d, int nx, int ny,
                                                int nz, const uint8_t* mat, const float* w,
                                                const float* kappa, const float* phi,
                                                const MatConst& mc, float* ks, float* as,
                                                float* bs)
{
    const int dx = c_dir[d][0], dy = c_dir[d][1], dz = c_dir[d][2];
    // Per axis: a non-zero offset fixes the voxel coordinate to the smaller corner coordinate;
    // a zero offset allows the two voxels on either side of the corner.
    int lo[3], hi[3];
    const int c0[3] = {ci, cj, ck};
    const int dd[3] = {dx, dy, dz};
    const int nn[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
        if (dd[a] != 0) {
            int v = dd[a] > 0 ? c0[a] : c0[a] - 1;
            lo[a] = v; hi[a] = v;
        } else {
            lo[a] = c0[a] - 1; hi[a] = c0[a];
        }
        if (lo[a] < 0) lo[a] = 0;
        if (hi[a] > nn[a] - 1) hi[a] = nn[a] - 1;
    }
    int n = 0;
    float k = 0.f, al = 0.f, be = 0.f;
    for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y)
            for (int x = lo[0]; x <= hi[0]; ++x) {
                int v = x + nx * (y + ny * z);
                int m = mat[v];
                if (m == 0) continue;
                ++n;
                if (ks) {
                    float s, c;
                    sincosf(phi[v], &s, &c);
                    float amp = w[v] * mc.amp[m];
                    k += w[v] * kappa[v];
                    al += amp * c;
                    be += amp * s;
                }
            }
    if (ks && n > 0) {
        float inv = 1.0f / (float)n;
        *ks = k * inv; *as = al * inv; *bs = be * inv;
    }
    return n;
}

__global__ void __launch_bounds__(kTopoThreads)
k_topology(PopView pv, const uint8_t* __restrict__ mat_raw_all, uint8_t* __restrict__ mat_all,
           const float* __restrict__ w_all, const float* __restrict__ kappa_all,
           const float* __restrict__ phi_all, MatConst mc, double edge, int* label_all,
           int* count_all, int* corner_mass_all, int* mass_corner_all, int2* spr_ab_all,
           float4* spr_p_all, float4* spr_pack_all, uint32_t* cflags_all, float* prm_all,
           float4* x0_all, float4* x_all, float4* v_all, double* x0c, int* status)
{
    __shared__ int sh_scan[32];
    __shared__ int sh_changed;
    __shared__ unsigned long long sh_best;
    __shared__ int sh_zmin;
    __shared__ double sh_sum[32];

    const int r = blockIdx.x;
    const int tid = threadIdx.x, T = blockDim.x;
    const int nx = pv.dims[3 * r], ny = pv.dims[3 * r + 1], nz = pv.dims[3 * r + 2];
    const int V = nx * ny * nz;
    const int cx = nx + 1, cy = ny + 1, cz = nz + 1;
    const int C = cx * cy * cz;
    const int64_t vo = pv.voff[r], mo = pv.moff[r], so = pv.soff[r];
    const uint8_t* mat_raw = mat_raw_all + vo;
    uint8_t* mat = mat_all + vo;
    const float* w = w_all + vo;
    const float* kappa = kappa_all + vo;
    const float* phi = phi_all + vo;
    int* label = label_all + vo;
    int* count = count_all + vo;
    int* corner_mass = corner_mass_all + mo;

    // 1. labels: own index for occupied voxels
    for (int v = tid; v < V; v += T) {
        label[v] = mat_raw[v] != 0 ? v : INT_MAX;
        count[v] = 0;
    }
    if (tid == 0) sh_best = 0ull;
    // 2. min-label propagation with pointer jumping; labels only decrease, so this terminates.
    int iter = 0;
    const int max_iter = 4 * V + 16;
    for (;;) {
        __syncthreads();
        if (tid == 0) sh_changed = 0;
        __syncthreads();
        int local = 0;
        for (int v = tid; v < V; v += T) {
            int m = label[v];
            if (m == INT_MAX) continue;
            int j = label[m];
            if (j < m) m = j;
            int i = v % nx, jj = (v / nx) % ny, k = v / (nx * ny);
            int u;
            if (i > 0 && (u = label[v - 1]) < m) m = u;
            if (i < nx - 1 && (u = label[v + 1]) < m) m = u;
            if (jj > 0 && (u = label[v - nx]) < m) m = u;
            if (jj < ny - 1 && (u = label[v + nx]) < m) m = u;
            if (k > 0 && (u = label[v - nx * ny]) < m) m = u;
            if (k < nz - 1 && (u = label[v + nx * ny]) < m) m = u;
            if (m < label[v]) { label[v] = m; local = 1; }
        }
        if (local) sh_changed = 1;
        __syncthreads();
        if (sh_changed == 0) break;
        if (++iter > max_iter) { if (tid == 0) atomicOr(status, 1); break; }
    }
    // 3. component sizes and the kept component
    for (int v = tid; v < V; v += T) {
        int l = label[v];
        if (l != INT_MAX) atomicAdd(&count[l], 1);
    }
    __syncthreads();
    for (int v = tid; v < V; v += T) {
        int c = count[v];
        if (c > 0) {
            unsigned long long key = ((unsigned long long)c << 32) | (unsigned)(0x7fffffff - v);
            atomicMax(&sh_best, key);
        }
    }
    __syncthreads();
    const int best = sh_best == 0ull ? -1 : 0x7fffffff - (int)(sh_best & 0xffffffffull);
    for (int v = tid; v < V; v += T) mat[v] = (best >= 0 && label[v] == best) ? mat_raw[v] : 0;
    for (int c = tid; c < C; c += T) corner_mass[c] = 0;
    __syncthreads();
    // 4. corners of kept voxels
    for (int v = tid; v < V; v += T) {
        if (mat[v] == 0) continue;
        int i = v % nx, j = (v / nx) % ny, k = v / (nx * ny);
        for (int d = 0; d < 8; ++d)
            corner_mass[(i + (d & 1)) + cx * ((j + ((d >> 1) & 1)) + cy * (k + ((d >> 2) & 1)))] = 1;
    }
    __syncthreads();
    // 5. mass indices in ascending corner order: each thread takes a contiguous chunk
    const int chunk = (C + T - 1) / T;
    const int c_beg = min(C, tid * chunk), c_end = min(C, c_beg + chunk);
    int cnt = 0;
    for (int c = c_beg; c < c_end; ++c) cnt += corner_mass[c];
    int M;
    int base = block_exclusive_scan(cnt, sh_scan, &M);
    int* mass_corner = mass_corner_all + mo;
    for (int c = c_beg; c < c_end; ++c) {
        if (corner_mass[c]) { corner_mass[c] = base; mass_corner[base] = c; ++base; }
        else corner_mass[c] = -1;
    }
    if (tid == 0) { sh_zmin = INT_MAX; pv.n_mass[r] = M; }
    __syncthreads();
    // 6. initial pose: lattice with the lowest mass at z = 0, at rest.  State is indexed by
    //    corner (all corners of the grid; corners without a mass carry no spring).  It is kept
    //    as the displacement u from this rest lattice (small, hence precise in float32), with
    //    the rest height z0 in the fourth lane: u = (ux, uy, uz, z0).
    for (int m = tid; m < M; m += T) atomicMin(&sh_zmin, mass_corner[m] / (cx * cy));
    __syncthreads();
    const int zmin = sh_zmin == INT_MAX ? 0 : sh_zmin;
    double xs = 0.0;
    for (int c = tid; c < C; c += T) {
        int ci = c % cx, cj = (c / cx) % cy, ck = c / (cx * cy);
        float4 p = make_float4((float)(ci * edge), (float)(cj * edge), (float)((ck - zmin) * edge), 0.f);
        x0_all[mo + c] = p;
        x_all[mo + c] = make_float4(0.f, 0.f, 0.f, p.z);
        v_all[mo + c] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (corner_mass[c] >= 0) xs += (double)p.x;
    }
    for (int o = 16; o > 0; o >>= 1) xs += __shfl_down_sync(0xffffffffu, xs, o);
    if ((tid & 31) == 0) sh_sum[tid >> 5] = xs;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int i = 0; i < (T + 31) / 32; ++i) t += sh_sum[i];
        x0c[r] = M > 0 ? t / M : 0.0;
    }
    // 7. springs: per mass (contiguous chunks), the 13 forward directions in corner-id order
    const int mchunk = (M + T - 1) / T;
    const int m_beg = min(M, tid * mchunk), m_end = min(M, m_beg + mchunk);
    int ns = 0;
    for (int m = m_beg; m < m_end; ++m) {
        int c = mass_corner[m];
        int ci = c % cx, cj = (c / cx) % cy, ck = c / (cx * cy);
        for (int d = 0; d < 13; ++d) {
            int bi = ci + c_dir[d][0], bj = cj + c_dir[d][1], bk = ck + c_dir[d][2];
            if (bi < 0 || bj < 0 || bi >= cx || bj >= cy || bk >= cz) continue;
            if (spring_incidence(ci, cj, ck, d, nx, ny, nz, mat, w, kappa, phi, mc, nullptr,
                                 nullptr, nullptr) > 0)
                ++ns;
        }
    }
    int S;
    int sbase = block_exclusive_scan(ns, sh_scan, &S);
    const double e1 = edge, e2 = edge * 1.4142135623730951, e3 = edge * 1.7320508075688772;
    for (int m = m_beg; m < m_end; ++m) {
        int c = mass_corner[m];
        int ci = c % cx, cj = (c / cx) % cy, ck = c / (cx * cy);
        for (int d = 0; d < 13; ++d) {
            int bi = ci + c_dir[d][0], bj = cj + c_dir[d][1], bk = ck + c_dir[d][2];
            if (bi < 0 || bj < 0 || bi >= cx || bj >= cy || bk >= cz) continue;
            float k, al, be;
            if (spring_incidence(ci, cj, ck, d, nx, ny, nz, mat, w, kappa, phi, mc, &k, &al,
                                 &be) == 0)
                continue;
            int b = corner_mass[bi + cx * (bj + cy * bk)];
            int cls = (c_dir[d][0] != 0) + (c_dir[d][1] != 0) + (c_dir[d][2] != 0);
            float L0 = (float)(cls == 1 ? e1 : (cls == 2 ? e2 : e3));
            spr_ab_all[so + sbase] = make_int2(m, b);
            spr_p_all[so + sbase] = make_float4(L0, k, al, be);
            ++sbase;
        }
    }
    if (tid == 0) pv.n_spring[r] = S;
    if (!cflags_all) return;
    // 9. the lattice kernel's tables, indexed by corner: forward-spring mask (bits 0..12),
    //    backward-spring mask (bits 16..28: a spring from corner c - offset(d) to c), mass bit 31,
    //    and the forward springs' (k, alpha L0, beta L0) as [3][13][C] planes.
    uint32_t* cflags = cflags_all + mo;
    float* prm = prm_all + 39 * mo;
    __syncthreads();
    for (int c = tid; c < C; c += T) {
        int ci = c % cx, cj = (c / cx) % cy, ck = c / (cx * cy);
        uint32_t fl = corner_mass[c] >= 0 ? 0x80000000u : 0u;
        for (int d = 0; d < 13; ++d) {
            float k = 0.f, al = 0.f, be = 0.f;
            int bi = ci + c_dir[d][0], bj = cj + c_dir[d][1], bk = ck + c_dir[d][2];
            if (corner_mass[c] >= 0 && bi >= 0 && bj >= 0 && bi < cx && bj < cy && bk < cz &&
                spring_incidence(ci, cj, ck, d, nx, ny, nz, mat, w, kappa, phi, mc, &k, &al, &be) > 0) {
                fl |= 1u << d;
                const int cls = (c_dir[d][0] != 0) + (c_dir[d][1] != 0) + (c_dir[d][2] != 0);
                const float L0 = (float)(cls == 1 ? e1 : (cls == 2 ? e2 : e3));
                al *= L0;
                be *= L0;
            } else {
                k = 0.f; al = 0.f; be = 0.f;
            }
            prm[(0 * 13 + d) * C + c] = k;
            prm[(1 * 13 + d) * C + c] = al;
            prm[(2 * 13 + d) * C + c] = be;
        }
        cflags[c] = fl;
    }
    __syncthreads();
    for (int c = tid; c < C; c += T) {
        int ci = c % cx, cj = (c / cx) % cy, ck = c / (cx * cy);
        uint32_t bw = 0;
        for (int d = 0; d < 13; ++d) {
            int ai = ci - c_dir[d][0], aj = cj - c_dir[d][1], ak = ck - c_dir[d][2];
            if (ai < 0 || aj < 0 || ak < 0 || ai >= cx || aj >= cy) continue;
            if ((cflags[ai + cx * (aj + cy * ak)] >> d) & 1u) bw |= 1u << (16 + d);
        }
        cflags[c] |= bw;
    }
    if (!spr_pack_all) return;
    __syncthreads();
    // 10. the atomic kernel's copy of the springs, direction-major (all springs of direction 0,
    //     then direction 1, ...), and within a direction interleaved over the residue of the
    //     corner id mod 32: round j holds the j-th spring (by ascending corner) of every residue
    //     that has one, in residue order.  Consecutive entries then have corners that differ mod
    //     32, so a warp's float atomics and float4 loads at either endpoint fall on distinct
    //     shared-memory banks, also in sparse robots, where ascending corners leave gaps.
    //     Packed as (k, alpha L0, beta L0, corner a | corner b << 14 | direction << 28) from the
    //     planes of step 9.  Warp w takes direction w, lane l the corners a = l (mod 32).
    __shared__ int sh_cnt[13][32];
    const int lane = tid & 31, warp = tid >> 5, nwarps = (T + 31) >> 5;
    for (int d = warp; d < 13; d += nwarps) {
        int cnt = 0;
        for (int a = lane; a < C; a += 32) cnt += (int)((cflags[a] >> d) & 1u);
        sh_cnt[d][lane] = cnt;
    }
    __syncthreads();
    float4* pack = spr_pack_all + so;
    for (int d = warp; d < 13; d += nwarps) {
        int dbase = 0;
        for (int e = 0; e < d; ++e)
            for (int b = 0; b < 32; ++b) dbase += sh_cnt[e][b];
        const int off = c_dir[d][0] + cx * (c_dir[d][1] + cy * c_dir[d][2]);
        int k = 0;                             // rank of this lane's next spring in its residue
        for (int a = lane; a < C; a += 32) {
            if (!((cflags[a] >> d) & 1u)) continue;
            int pos = dbase;                   // springs of earlier rounds, then earlier residues
            for (int b = 0; b < 32; ++b) {
                const int nb = sh_cnt[d][b];
                pos += min(nb, k) + ((b < lane && nb > k) ? 1 : 0);
            }
            const unsigned bits = (unsigned)a | ((unsigned)(a + off) << 14) | ((unsigned)d << 28);
            pack[pos] = make_float4(prm[d * C + a], prm[(13 + d) * C + a], prm[(26 + d) * C + a],
                                    __uint_as_float(bits));
            ++k;
        }
    }
}

}  // namespace

cudaError_t launch_topology(PopView pv, const uint8_t* mat_raw, uint8_t* mat, const float* w,
                            const float* kappa, const float* phi, MatConst mc, double edge,
                            int* label, int* count, int* corner_mass, int* mass_corner,
                            int2* spr_ab, float4* spr_p, float4* spr_pack, uint32_t* cflags,
                            float* prm, float4* x0, float4* x, float4* v, double* x0c, int* status,
                            int max_threads, cudaStream_t s)
{
    if (pv.P == 0) return cudaSuccess;
    int T = max_threads > 0 && max_threads < kTopoThreads ? max_threads : kTopoThreads;
    k_topology<<<pv.P, T, 0, s>>>(pv, mat_raw, mat, w, kappa, phi, mc, edge, label, count,
                                  corner_mass, mass_corner, spr_ab, spr_p, spr_pack, cflags, prm,
                                  x0, x, v, x0c, status);
    return cudaGetLastError();
}

}  // namespace vx
