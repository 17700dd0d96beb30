// sem_mesh.cu -- mesh construction: GLL data (host), box connectivity and
// gather-scatter groups (host), geometric factors, mass, multiplicity and
// the assembled Jacobi diagonal (device).
//
// Paper: section 3.1 -- E hexahedral elements, order-N Lagrange basis on the
// GLL points, unit-depth gather-scatter over shared nodes.  Formulas: the
// textbook SEM the paper cites (Deville, Fischer & Mund 2002).

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "sem_common.cuh"

namespace sem {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return SEM_ERR_CUDA;
}

// ---------------------------------------------------------------- GLL (host)

// GLL points are -1, +1 and the zeros of q(x) = x P_N(x) - P_{N-1}(x) on the
// open interval (q is proportional to (1-x^2) P_N'(x)); q'(x) = (N+1) P_N(x).
// Newton from the Chebyshev-Gauss-Lobatto points.  Weights 2/(N(N+1)P_N^2).
static void legendre_pair(int N, double x, double *PN, double *PNm1) {
    double a = 1.0, b = x;  // P_0, P_1
    if (N == 0) { *PN = 1.0; *PNm1 = 0.0; return; }
    for (int k = 2; k <= N; ++k) {
        double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
        a = b;
        b = c;
    }
    *PN = b;
    *PNm1 = a;
}

void gll_host(int N, double *xi, double *rho) {
    for (int i = 0; i <= N; ++i) {
        double x = -std::cos(M_PI * i / N);
        if (i > 0 && i < N) {
            for (int it = 0; it < 200; ++it) {
                double P, Pm;
                legendre_pair(N, x, &P, &Pm);
                double dx = (x * P - Pm) / ((N + 1) * P);
                x -= dx;
                if (std::fabs(dx) <= 1e-16) break;
            }
        }
        xi[i] = x;
    }
    for (int i = 0; i < (N + 1) / 2; ++i) {  // exact symmetry
        double s = 0.5 * (xi[N - i] - xi[i]);
        xi[i] = -s;
        xi[N - i] = s;
    }
    if (N % 2 == 0) xi[N / 2] = 0.0;
    for (int i = 0; i <= N; ++i) {
        double P, Pm;
        legendre_pair(N, xi[i], &P, &Pm);
        rho[i] = 2.0 / (N * (N + 1.0) * P * P);
    }
}

// D_ij = l_j'(xi_i) by the barycentric formula: lambda_j = 1/prod_{k!=j}(x_j-x_k),
// D_ij = (lambda_j/lambda_i)/(x_i-x_j), D_ii = -sum_{j!=i} D_ij.
void deriv_host(int N, const double *x, double *D) {
    const int n1 = N + 1;
    double lam[kMaxN1];
    for (int j = 0; j < n1; ++j) {
        double p = 1.0;
        for (int k = 0; k < n1; ++k)
            if (k != j) p *= (x[j] - x[k]);
        lam[j] = 1.0 / p;
    }
    for (int i = 0; i < n1; ++i) {
        double s = 0.0;
        for (int j = 0; j < n1; ++j) {
            if (j == i) continue;
            double d = (lam[j] / lam[i]) / (x[i] - x[j]);
            D[i * n1 + j] = d;
            s += d;
        }
        D[i * n1 + i] = -s;
    }
}

// ---------------------------------------------------------------- connectivity (host)

// Per axis: for each 1-D global index I, the list of (element coordinate,
// local index) copies, and whether I lies on a Dirichlet end.
struct Axis {
    int64_t G;                              // number of 1-D global indices
    std::vector<int> start, cnt;            // copies of I: pairs[start[I] .. +cnt[I])
    std::vector<std::pair<int, int>> pairs; // (e_a, i)
    std::vector<char> dir;                  // Dirichlet end flag
};

static Axis make_axis(int N, int nel, int periodic, int lo_dir, int hi_dir) {
    Axis a;
    a.G = (int64_t)nel * N + (periodic ? 0 : 1);
    std::vector<std::vector<std::pair<int, int>>> tmp(a.G);
    for (int e = 0; e < nel; ++e)
        for (int i = 0; i <= N; ++i) {
            int64_t I = (int64_t)e * N + i;
            if (periodic) I %= a.G;
            tmp[I].push_back({e, i});
        }
    a.start.resize(a.G);
    a.cnt.resize(a.G);
    a.dir.assign(a.G, 0);
    for (int64_t I = 0; I < a.G; ++I) {
        a.start[I] = (int)a.pairs.size();
        a.cnt[I] = (int)tmp[I].size();
        for (auto &p : tmp[I]) a.pairs.push_back(p);
    }
    if (!periodic) {
        if (lo_dir) a.dir[0] = 1;
        if (hi_dir) a.dir[a.G - 1] = 1;
    }
    return a;
}

// Groups: every global node with more than one copy, or on a Dirichlet face.
// Group sizes are products of per-axis copy counts (1 or 2): 1, 2, 4 or 8.
// They are stored in four buckets by size (bucket b holds groups of 2^b
// copies, size-1 groups only when masked), each bucket's masked groups first,
// then the rest, each part in lexicographic (I fastest) order of the global
// node; each bucket starts on a 16-byte boundary.
struct GsCounts {
    int64_t ngroups = 0, nmasked = 0, nentries = 0;
    int64_t n[4] = {0, 0, 0, 0}, nm[4] = {0, 0, 0, 0}, start[4] = {0, 0, 0, 0};
    int64_t ints = 0;  // length of the bucketed index array (with padding)
};

static int bucket_of(int m) { return m == 1 ? 0 : m == 2 ? 1 : m == 4 ? 2 : 3; }

static GsCounts gs_count(const Axis ax[3]) {
    // histogram over (copies, dirichlet) per axis, product over axes
    GsCounts c;
    int64_t h[3][3][2] = {};
    for (int a = 0; a < 3; ++a)
        for (int64_t I = 0; I < ax[a].G; ++I) h[a][ax[a].cnt[I]][ax[a].dir[I]]++;
    for (int mx = 1; mx <= 2; ++mx)
        for (int my = 1; my <= 2; ++my)
            for (int mz = 1; mz <= 2; ++mz)
                for (int dx = 0; dx < 2; ++dx)
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dz = 0; dz < 2; ++dz) {
                            int64_t n = h[0][mx][dx] * h[1][my][dy] * h[2][mz][dz];
                            if (!n) continue;
                            int m = mx * my * mz;
                            bool masked = dx || dy || dz;
                            if (m < 2 && !masked) continue;
                            c.ngroups += n;
                            c.nentries += n * m;
                            c.n[bucket_of(m)] += n;
                            if (masked) {
                                c.nmasked += n;
                                c.nm[bucket_of(m)] += n;
                            }
                        }
    int64_t at = 0;
    for (int b = 0; b < 4; ++b) {
        c.start[b] = at;
        at += c.n[b] << b;
        at = (at + 3) / 4 * 4;
    }
    c.ints = at;
    return c;
}

static void gs_build(const Axis ax[3], int N, const int nel[3], const GsCounts &c, std::vector<int> &idx) {
    const int n1 = N + 1;
    const int64_t npt = (int64_t)n1 * n1 * n1;
    idx.assign(c.ints > 0 ? c.ints : 1, 0);
    int64_t cur[4];
    for (int b = 0; b < 4; ++b) cur[b] = c.start[b];
    for (int pass = 0; pass < 2; ++pass) {  // pass 0: masked groups, pass 1: the rest
        for (int64_t K = 0; K < ax[2].G; ++K)
            for (int64_t J = 0; J < ax[1].G; ++J)
                for (int64_t I = 0; I < ax[0].G; ++I) {
                    int cx = ax[0].cnt[I], cy = ax[1].cnt[J], cz = ax[2].cnt[K];
                    bool masked = ax[0].dir[I] || ax[1].dir[J] || ax[2].dir[K];
                    int m = cx * cy * cz;
                    if (masked != (pass == 0)) continue;
                    if (!masked && m < 2) continue;
                    int loc[8], n = 0;
                    for (int c2 = 0; c2 < cz; ++c2)
                        for (int c1 = 0; c1 < cy; ++c1)
                            for (int c0 = 0; c0 < cx; ++c0) {
                                auto px = ax[0].pairs[ax[0].start[I] + c0];
                                auto py = ax[1].pairs[ax[1].start[J] + c1];
                                auto pz = ax[2].pairs[ax[2].start[K] + c2];
                                int64_t e = px.first + (int64_t)nel[0] * (py.first + (int64_t)nel[1] * pz.first);
                                loc[n++] = (int)(e * npt + px.second + n1 * (py.second + n1 * pz.second));
                            }
                    // ascending local index: the summation order of every group
                    for (int s = 1; s < n; ++s)
                        for (int t = s; t > 0 && loc[t - 1] > loc[t]; --t) std::swap(loc[t - 1], loc[t]);
                    int64_t &q = cur[bucket_of(n)];
                    for (int s = 0; s < n; ++s) idx[q++] = loc[s];
                }
    }
}

static int validate(const sem_mesh_desc *d) {
    if (!d) return fail(SEM_ERR_INVALID_ARG, "desc is NULL");
    if (d->N < 1 || d->N > kMaxN) return fail(SEM_ERR_UNSUPPORTED, "order N out of range 1..SEM_MAX_ORDER");
    for (int a = 0; a < 3; ++a)
        if (d->nel[a] < 1) return fail(SEM_ERR_INVALID_ARG, "nel must be >= 1");
    if (!d->vertices) return fail(SEM_ERR_INVALID_ARG, "vertices is NULL");
    int64_t E = (int64_t)d->nel[0] * d->nel[1] * d->nel[2];
    int64_t nloc = E * (d->N + 1) * (d->N + 1) * (d->N + 1);
    if (nloc >= (int64_t(1) << 31)) return fail(SEM_ERR_INVALID_ARG, "E*(N+1)^3 must be < 2^31");
    if (d->geom_flags & ~(SEM_GEOM_F32 | SEM_GEOM_RX | SEM_GEOM_PAIR | SEM_GEOM_AFFINE | SEM_GEOM_BF16))
        return fail(SEM_ERR_INVALID_ARG, "unknown geom_flags bit");
    if ((d->geom_flags & SEM_GEOM_BF16) && !(d->geom_flags & SEM_GEOM_F32))
        return fail(SEM_ERR_INVALID_ARG, "SEM_GEOM_BF16 needs SEM_GEOM_F32");
    if ((d->geom_flags & SEM_GEOM_AFFINE) && !(d->geom_flags & SEM_GEOM_F32))
        return fail(SEM_ERR_INVALID_ARG, "SEM_GEOM_AFFINE needs SEM_GEOM_F32");
    return SEM_OK;
}

struct Layout {
    size_t verts, G, G32, G2, aff, G16, B, mult, minv, dinv, dinv32, minv32, rx, idx, err, total;
};

static Layout layout_for(const sem_mesh_desc *d, const GsCounts &c) {
    const int64_t E = (int64_t)d->nel[0] * d->nel[1] * d->nel[2];
    const int64_t npt = (int64_t)(d->N + 1) * (d->N + 1) * (d->N + 1);
    const int64_t nloc = E * npt;
    const bool f32 = d->geom_flags & SEM_GEOM_F32;
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes); return at; };
    L.verts = take(sizeof(double) * E * 24);
    L.G = take(sizeof(double) * E * 6 * npt);
    L.G32 = f32 ? take(sizeof(float) * E * 6 * npt) : 0;
    L.G2 = (d->geom_flags & SEM_GEOM_PAIR) ? take(sizeof(float2) * E * 6 * npt) : 0;
    L.aff = (d->geom_flags & SEM_GEOM_AFFINE) ? take(sizeof(float) * 4 * E) : 0;
    L.G16 = (d->geom_flags & SEM_GEOM_BF16) ? take(sizeof(__nv_bfloat16) * E * 6 * npt) : 0;
    L.B = take(sizeof(double) * nloc);
    L.mult = take(sizeof(double) * nloc);
    L.minv = take(sizeof(double) * nloc);
    L.dinv = take(sizeof(double) * nloc);
    L.dinv32 = f32 ? take(sizeof(float) * nloc) : 0;
    L.minv32 = f32 ? take(sizeof(float) * nloc) : 0;
    L.rx = (d->geom_flags & SEM_GEOM_RX) ? take(sizeof(double) * 9 * nloc) : 0;
    L.idx = take(sizeof(int) * (c.ints > 0 ? c.ints : 1));
    L.err = take(sizeof(int) * 8);
    L.total = o;
    return L;
}

static void make_axes(const sem_mesh_desc *d, Axis ax[3]) {
    for (int a = 0; a < 3; ++a)
        ax[a] = make_axis(d->N, d->nel[a], d->periodic[a] != 0, (d->dirichlet_faces >> (2 * a)) & 1,
                          (d->dirichlet_faces >> (2 * a + 1)) & 1);
}

// ---------------------------------------------------------------- device kernels

struct GllConst {
    double xi[kMaxN1], rho[kMaxN1];
};

// Geometric factors of trilinear hexahedra, one thread per local point.  The
// Jacobian J_ab = dx_a/dr_b is the analytic derivative of the trilinear map.
__global__ void geometry_kernel(const double *__restrict__ verts, int64_t E, int N, GllConst g,
                                double *__restrict__ G, double *__restrict__ B,
                                float *__restrict__ G32, double *__restrict__ rx, int *__restrict__ err) {
    const int n1 = N + 1;
    const int64_t npt = (int64_t)n1 * n1 * n1;
    const int64_t nloc = E * npt;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nloc;
         l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = l / npt;
        const int p = (int)(l - e * npt);
        const int i = p % n1, j = (p / n1) % n1, k = p / (n1 * n1);
        const double r = g.xi[i], s = g.xi[j], t = g.xi[k];
        const double fr[2] = {0.5 * (1.0 - r), 0.5 * (1.0 + r)};
        const double fs[2] = {0.5 * (1.0 - s), 0.5 * (1.0 + s)};
        const double ft[2] = {0.5 * (1.0 - t), 0.5 * (1.0 + t)};
        const double df[2] = {-0.5, 0.5};
        double J[3][3] = {};
        const double *V = verts + e * 24;
        // vertex offsets from vertex 0: the derivative is unchanged and the
        // sum cancels less when the element lies far from the origin
        for (int v = 1; v < 8; ++v) {
            const int bx = v & 1, by = (v >> 1) & 1, bz = (v >> 2) & 1;
            const double gr = df[bx] * fs[by] * ft[bz];
            const double gs = fr[bx] * df[by] * ft[bz];
            const double gt = fr[bx] * fs[by] * df[bz];
            for (int a = 0; a < 3; ++a) {
                const double X = V[v * 3 + a] - V[a];
                J[a][0] += X * gr;
                J[a][1] += X * gs;
                J[a][2] += X * gt;
            }
        }
        // cofactors C[a][b]; inverse (J^-1)[b][a] = C[a][b] / det
        double C[3][3];
        C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
        if (!(det > 0.0)) atomicAdd(err + 1, 1);
        // dr_b/dx_a = C[a][b] / det  ->  G_bc = wq sum_a (C[a][b] C[a][c]) / det^2
        const double wq = g.rho[i] * g.rho[j] * g.rho[k];
        const double sc = wq / det;
        double gg[6];
        gg[0] = sc * (C[0][0] * C[0][0] + C[1][0] * C[1][0] + C[2][0] * C[2][0]);
        gg[1] = sc * (C[0][1] * C[0][1] + C[1][1] * C[1][1] + C[2][1] * C[2][1]);
        gg[2] = sc * (C[0][2] * C[0][2] + C[1][2] * C[1][2] + C[2][2] * C[2][2]);
        gg[3] = sc * (C[0][0] * C[0][1] + C[1][0] * C[1][1] + C[2][0] * C[2][1]);
        gg[4] = sc * (C[0][0] * C[0][2] + C[1][0] * C[1][2] + C[2][0] * C[2][2]);
        gg[5] = sc * (C[0][1] * C[0][2] + C[1][1] * C[1][2] + C[2][1] * C[2][2]);
        double *Ge = G + e * 6 * npt;
        for (int c = 0; c < 6; ++c) Ge[c * npt + p] = gg[c];
        if (G32) {
            float *Gf = G32 + e * 6 * npt;
            for (int c = 0; c < 6; ++c) Gf[c * npt + p] = (float)gg[c];
        }
        B[l] = wq * det;
        if (rx) {
            // dr_a/dx_m = (J^-1)[a][m] = C[m][a] / det, stored [e][3a+m][p]
            double *Re = rx + e * 9 * npt;
            const double id = 1.0 / det;
            for (int a = 0; a < 3; ++a)
                for (int mm = 0; mm < 3; ++mm) Re[(3 * a + mm) * npt + p] = C[mm][a] * id;
        }
    }
}

__global__ void coords_kernel(const double *__restrict__ verts, int64_t E, int N, GllConst g,
                              double *__restrict__ xyz) {
    const int n1 = N + 1;
    const int64_t npt = (int64_t)n1 * n1 * n1;
    const int64_t nloc = E * npt;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nloc;
         l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = l / npt;
        const int p = (int)(l - e * npt);
        const int i = p % n1, j = (p / n1) % n1, k = p / (n1 * n1);
        const double f[3][2] = {{0.5 * (1 - g.xi[i]), 0.5 * (1 + g.xi[i])},
                                {0.5 * (1 - g.xi[j]), 0.5 * (1 + g.xi[j])},
                                {0.5 * (1 - g.xi[k]), 0.5 * (1 + g.xi[k])}};
        const double *V = verts + e * 24;
        for (int a = 0; a < 3; ++a) {
            double x = 0.0;
            for (int v = 0; v < 8; ++v) x += V[v * 3 + a] * (f[0][v & 1] * f[1][(v >> 1) & 1] * f[2][(v >> 2) & 1]);
            xyz[a * nloc + l] = x;
        }
    }
}

__global__ void fill_kernel(double *__restrict__ a, int64_t n, double v) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        a[l] = v;
}

// minv = 1/mult; dinv = 1/diag (the Dirichlet entries are zeroed afterwards
// by a mask-only gather-scatter pass); FP32 copies when requested.
__global__ void invert_kernel(const double *__restrict__ mult, double *__restrict__ minv,
                              double *__restrict__ dinv, float *__restrict__ minv32,
                              float *__restrict__ dinv32, int64_t n) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const double mi = 1.0 / mult[l];
        minv[l] = mi;
        const double di = 1.0 / dinv[l];
        dinv[l] = di;
        if (minv32) minv32[l] = (float)mi;
        if (dinv32) dinv32[l] = (float)di;
    }
}

// FP32-pair copy of the geometric factors: g = hi + lo with hi the nearest
// float and lo the nearest float to the remainder (48 significant bits).
__global__ void split_pair_kernel(const double *__restrict__ a, float2 *__restrict__ b, int64_t n) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const double g = a[l];
        const float hi = (float)g;
        b[l] = make_float2(hi, (float)(g - (double)hi));
    }
}

// BF16 copy (round to nearest even) of the geometric factors.
__global__ void to_bf16_kernel(const double *__restrict__ a, __nv_bfloat16 *__restrict__ b, int64_t n) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        b[l] = __float2bfloat16_rn((float)a[l]);
}

__global__ void copy_f32_from_f64(const double *__restrict__ a, float *__restrict__ b, int64_t n) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        b[l] = (float)a[l];
}

__global__ void gather_field_kernel(const double *__restrict__ src, int64_t E, int npt, int stride_e,
                                    int off, double *__restrict__ dst) {
    const int64_t n = E * npt;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = l / npt;
        dst[l] = src[e * stride_e + off + (l - e * npt)];
    }
}

static int grid_for(int64_t n, int block = 256) {
    int64_t g = (n + block - 1) / block;
    if (g > 152 * 64) g = 152 * 64;
    return (int)(g < 1 ? 1 : g);
}

// Self-test of the bounded waits: kind 0, one CTA waits on an mbarrier
// whose 16 transaction bytes no copy will bring (the wait of every bulk-copy
// pipeline of the library); kind 1, two CTAs wait on a grid barrier whose
// target exceeds the grid (the wait of the cooperative coarse solve).  Both
// give up after limit_ns, record their code in the error word and return;
// nothing is in flight when they exit.
__global__ void wait_selftest_kernel(int kind, uint64_t limit_ns, unsigned *ctr, int *err) {
    if (kind == 0) {
        __shared__ __align__(8) uint64_t bar;
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16);
        __syncthreads();
        mbar_wait_bounded(&bar, 0, err, kDevTimeoutTma, limit_ns);
    } else {
        grid_barrier_bounded(ctr, gridDim.x + 1, err, limit_ns);
    }
}

}  // namespace sem

using namespace sem;

extern "C" {

const char *sem_version(void) { return "sem_gb300 0.1 (sm_103a)"; }

const char *sem_last_error(void) { return g_last_error.c_str(); }

const char *sem_status_string(int s) {
    switch (s) {
        case SEM_OK: return "ok";
        case SEM_ERR_INVALID_ARG: return "invalid argument";
        case SEM_ERR_CUDA: return "CUDA error";
        case SEM_ERR_MESH: return "bad mesh (det J <= 0)";
        case SEM_ERR_WORKSPACE: return "workspace too small or misaligned";
        case SEM_ERR_NAN: return "NaN or Inf in right-hand side";
        case SEM_ERR_NOT_CONVERGED: return "not converged";
        case SEM_ERR_TIMEOUT: return "device wait timed out";
        case SEM_ERR_UNSUPPORTED: return "unsupported order or option";
        default: return "unknown status";
    }
}

size_t sem_mesh_workspace_bytes(const sem_mesh_desc *d) {
    if (validate(d) != SEM_OK) return 0;
    Axis ax[3];
    make_axes(d, ax);
    return layout_for(d, gs_count(ax)).total;
}

int sem_mesh_create(const sem_mesh_desc *d, void *ws, size_t bytes, void *stream, sem_mesh **out) {
    int st = validate(d);
    if (st != SEM_OK) return st;
    if (!out) return fail(SEM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign))
        return fail(SEM_ERR_WORKSPACE, "workspace NULL or not 256-byte aligned");
    Axis ax[3];
    make_axes(d, ax);
    GsCounts c = gs_count(ax);
    Layout L = layout_for(d, c);
    if (bytes < L.total) return fail(SEM_ERR_WORKSPACE, "workspace smaller than sem_mesh_workspace_bytes");
    if (c.ints >= (int64_t(1) << 31)) return fail(SEM_ERR_INVALID_ARG, "too many shared points");

    sem_mesh *m = new (std::nothrow) sem_mesh();
    if (!m) return fail(SEM_ERR_INVALID_ARG, "host allocation failed");
    m->N = d->N;
    m->n1 = d->N + 1;
    m->npt = m->n1 * m->n1 * m->n1;
    m->E = (int64_t)d->nel[0] * d->nel[1] * d->nel[2];
    m->nloc = m->E * m->npt;
    for (int a = 0; a < 3; ++a) {
        m->nel[a] = d->nel[a];
        m->periodic[a] = d->periodic[a] != 0;
    }
    m->faces = d->dirichlet_faces;
    m->nglob = ax[0].G * ax[1].G * ax[2].G;
    m->geom_flags = d->geom_flags;
    m->ngroups = c.ngroups;
    m->nmasked = c.nmasked;
    m->nentries = c.nentries;
    for (int b = 0; b < 4; ++b) {
        m->gs_n[b] = c.n[b];
        m->gs_nm[b] = c.nm[b];
        m->gs_start[b] = c.start[b];
    }
    m->ws_bytes = L.total;
    gll_host(m->N, m->xi, m->rho);
    std::memset(&m->D, 0, sizeof(m->D));
    std::memset(&m->Df, 0, sizeof(m->Df));
    deriv_host(m->N, m->xi, m->D.d);
    for (int q = 0; q < m->n1 * m->n1; ++q) m->Df.d[q] = (float)m->D.d[q];

    char *base = static_cast<char *>(ws);
    m->verts = reinterpret_cast<double *>(base + L.verts);
    m->G = reinterpret_cast<double *>(base + L.G);
    m->G32 = (d->geom_flags & SEM_GEOM_F32) ? reinterpret_cast<float *>(base + L.G32) : nullptr;
    m->G2 = (d->geom_flags & SEM_GEOM_PAIR) ? reinterpret_cast<float2 *>(base + L.G2) : nullptr;
    m->aff32 = (d->geom_flags & SEM_GEOM_AFFINE) ? reinterpret_cast<float *>(base + L.aff) : nullptr;
    m->G16 = (d->geom_flags & SEM_GEOM_BF16) ? static_cast<void *>(base + L.G16) : nullptr;
    m->B = reinterpret_cast<double *>(base + L.B);
    m->mult = reinterpret_cast<double *>(base + L.mult);
    m->minv = reinterpret_cast<double *>(base + L.minv);
    m->dinv = reinterpret_cast<double *>(base + L.dinv);
    m->dinv32 = m->G32 ? reinterpret_cast<float *>(base + L.dinv32) : nullptr;
    m->minv32 = m->G32 ? reinterpret_cast<float *>(base + L.minv32) : nullptr;
    m->rx = (d->geom_flags & SEM_GEOM_RX) ? reinterpret_cast<double *>(base + L.rx) : nullptr;
    m->gs_idx = reinterpret_cast<int *>(base + L.idx);
    m->d_err = reinterpret_cast<int *>(base + L.err);

    auto cleanup = [&](int code) {
        delete m;
        return code;
    };
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cleanup(cuda_fail(ce, "cudaGetDevice"));
    m->device = dev;
    ce = cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) return cleanup(cuda_fail(ce, "cudaDeviceGetAttribute"));

    std::vector<int> idx;
    gs_build(ax, m->N, m->nel, c, idx);
    cudaStream_t s = as_stream(stream);
#define CK(call)                                              \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return cleanup(cuda_fail(_e, #call)); \
    } while (0)
    CK(cudaMemcpyAsync(m->verts, d->vertices, sizeof(double) * m->E * 24, cudaMemcpyHostToDevice, s));
    std::vector<float> aff;
    if (m->aff32) {
        // axis-aligned boxes: vertex v = V0 + (vx hx, vy hy, vz hz); then J =
        // diag(h)/2, det J = hx hy hz / 8 and G_rr = rho_i rho_j rho_k hy hz / (2 hx),
        // G_ss = ... hx hz / (2 hy), G_tt = ... hx hy / (2 hz), cross terms 0
        aff.resize(4 * m->E);
        for (int64_t e = 0; e < m->E; ++e) {
            const double *V = d->vertices + e * 24;
            const double h[3] = {V[1 * 3 + 0] - V[0], V[2 * 3 + 1] - V[1], V[4 * 3 + 2] - V[2]};
            const double tol = 1e-12 * (std::fabs(h[0]) + std::fabs(h[1]) + std::fabs(h[2]));
            bool ok = h[0] > 0 && h[1] > 0 && h[2] > 0;
            for (int v = 0; v < 8 && ok; ++v) {
                const int b[3] = {v & 1, (v >> 1) & 1, (v >> 2) & 1};
                for (int a = 0; a < 3; ++a)
                    if (std::fabs(V[v * 3 + a] - (V[a] + b[a] * h[a])) > tol) ok = false;
            }
            if (!ok) {
                delete m;
                return fail(SEM_ERR_MESH, "SEM_GEOM_AFFINE: element " + std::to_string(e) +
                                              " is not an axis-aligned box");
            }
            aff[4 * e + 0] = (float)(h[1] * h[2] / (2.0 * h[0]));
            aff[4 * e + 1] = (float)(h[0] * h[2] / (2.0 * h[1]));
            aff[4 * e + 2] = (float)(h[0] * h[1] / (2.0 * h[2]));
            aff[4 * e + 3] = 0.f;
        }
        CK(cudaMemcpyAsync(m->aff32, aff.data(), sizeof(float) * aff.size(), cudaMemcpyHostToDevice, s));
    }
    CK(cudaMemcpyAsync(m->gs_idx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(m->d_err, 0, sizeof(int) * 8, s));
    GllConst g{};
    for (int i = 0; i < m->n1; ++i) {
        g.xi[i] = m->xi[i];
        g.rho[i] = m->rho[i];
    }
    geometry_kernel<<<grid_for(m->nloc), 256, 0, s>>>(m->verts, m->E, m->N, g, m->G, m->B, m->G32, m->rx,
                                                      m->d_err);
    CK(cudaGetLastError());
    if (m->G2) {
        split_pair_kernel<<<grid_for(m->E * 6 * m->npt), 256, 0, s>>>(m->G, m->G2, m->E * 6 * m->npt);
        CK(cudaGetLastError());
    }
    if (m->G16) {
        to_bf16_kernel<<<grid_for(m->E * 6 * m->npt), 256, 0, s>>>(m->G, static_cast<__nv_bfloat16 *>(m->G16),
                                                                   m->E * 6 * m->npt);
        CK(cudaGetLastError());
    }
    // multiplicity = Q Q^T 1
    fill_kernel<<<grid_for(m->nloc), 256, 0, s>>>(m->mult, m->nloc, 1.0);
    CK(cudaGetLastError());
    st = gs_launch(m, m->mult, SEM_F64, kGsSum, s);
    if (st != SEM_OK) return cleanup(st);
    // assembled Jacobi diagonal Q Q^T diag(A_L), inverted, 0 on Dirichlet nodes
    st = jacobi_diag_launch(m, m->dinv, s);
    if (st != SEM_OK) return cleanup(st);
    st = gs_launch(m, m->dinv, SEM_F64, kGsSum, s);
    if (st != SEM_OK) return cleanup(st);
    invert_kernel<<<grid_for(m->nloc), 256, 0, s>>>(m->mult, m->minv, m->dinv, nullptr, nullptr, m->nloc);
    CK(cudaGetLastError());
    st = gs_launch(m, m->dinv, SEM_F64, kGsMaskOnly, s);
    if (st != SEM_OK) return cleanup(st);
    if (m->G32) {
        copy_f32_from_f64<<<grid_for(m->nloc), 256, 0, s>>>(m->dinv, m->dinv32, m->nloc);
        CK(cudaGetLastError());
        copy_f32_from_f64<<<grid_for(m->nloc), 256, 0, s>>>(m->minv, m->minv32, m->nloc);
        CK(cudaGetLastError());
    }
    int herr[8];
    CK(cudaMemcpyAsync(herr, m->d_err, sizeof(herr), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
#undef CK
    if (herr[1] != 0) {
        delete m;
        return fail(SEM_ERR_MESH, "det J <= 0 at " + std::to_string(herr[1]) + " GLL points");
    }
    *out = m;
    return SEM_OK;
}

int sem_mesh_destroy(sem_mesh *m) {
    delete m;
    return SEM_OK;
}

int sem_mesh_get_info(const sem_mesh *m, sem_mesh_info *info) {
    if (!m || !info) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    info->N = m->N;
    info->E = m->E;
    info->nloc = m->nloc;
    info->nglob = m->nglob;
    info->n_paper = m->E * (int64_t)m->N * m->N * m->N;
    info->n_shared_groups = m->ngroups;
    info->n_shared_points = m->nentries;
    info->workspace_bytes = m->ws_bytes;
    return SEM_OK;
}

int sem_mesh_coords(const sem_mesh *m, double *xyz, void *stream) {
    if (!m || !xyz) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    GllConst g{};
    for (int i = 0; i < m->n1; ++i) {
        g.xi[i] = m->xi[i];
        g.rho[i] = m->rho[i];
    }
    coords_kernel<<<grid_for(m->nloc), 256, 0, as_stream(stream)>>>(m->verts, m->E, m->N, g, xyz);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

int sem_mesh_field(const sem_mesh *m, int which, double *dst, void *stream) {
    if (!m || !dst) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = as_stream(stream);
    const double *src = nullptr;
    switch (which) {
        case 0: src = m->B; break;
        case 1: src = m->mult; break;
        case 2: src = m->dinv; break;
        default:
            if (which >= 3 && which <= 8) {
                gather_field_kernel<<<grid_for(m->nloc), 256, 0, s>>>(m->G, m->E, m->npt, 6 * m->npt,
                                                                      (which - 3) * m->npt, dst);
                SEM_CUDA_CHECK(cudaGetLastError());
                return SEM_OK;
            }
            return fail(SEM_ERR_INVALID_ARG, "unknown field");
    }
    SEM_CUDA_CHECK(cudaMemcpyAsync(dst, src, sizeof(double) * m->nloc, cudaMemcpyDeviceToDevice, s));
    return SEM_OK;
}

int sem_wait_selftest(const sem_mesh *m, int kind, double limit_s, void *d_scratch, size_t bytes, void *stream) {
    if (!m) return fail(SEM_ERR_INVALID_ARG, "NULL mesh");
    if (kind != 0 && kind != 1) return fail(SEM_ERR_INVALID_ARG, "kind must be 0 (mbarrier) or 1 (grid barrier)");
    if (!(limit_s > 0.0) || limit_s > 10.0) return fail(SEM_ERR_INVALID_ARG, "limit_s must be in (0, 10]");
    if (kind == 1 && (!d_scratch || bytes < 16 || reinterpret_cast<uintptr_t>(d_scratch) % 16))
        return fail(SEM_ERR_WORKSPACE, "the grid-barrier self-test needs 16 bytes of aligned device scratch");
    cudaStream_t st = as_stream(stream);
    unsigned *ctr = static_cast<unsigned *>(d_scratch);
    if (kind == 1) SEM_CUDA_CHECK(cudaMemsetAsync(ctr, 0, sizeof(unsigned), st));
    wait_selftest_kernel<<<kind == 0 ? 1 : 2, 32, 0, st>>>(kind, (uint64_t)(limit_s * 1e9), ctr, m->d_err);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

int sem_mesh_check_device_error(const sem_mesh *m, int *code, void *stream) {
    if (!m || !code) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = as_stream(stream);
    int h = 0;
    SEM_CUDA_CHECK(cudaMemcpyAsync(&h, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    SEM_CUDA_CHECK(cudaStreamSynchronize(s));
    SEM_CUDA_CHECK(cudaMemsetAsync(m->d_err, 0, sizeof(int), s));
    *code = h;
    return SEM_OK;
}

}  // extern "C"
