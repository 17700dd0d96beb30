// sem_schwarz.cu -- hybrid Schwarz preconditioner of the pressure solve.
//
// Paper section 3.1: the pressure is solved by a Krylov method with a
// hybrid-Schwarz multigrid preconditioner (the SEM overlapping Schwarz /
// fast-diagonalisation method of the literature it cites).  Two additive
// levels, symmetric:
//   z = sum_e R_e^T A_e^{-1} R_e r  +  P A_c^{-1} P^T r.
// Local solves: element e extended by one GLL point into each neighbour
// (N+3 points per direction); along each direction the 1-D stiffness and mass
// of the three elements (left neighbour, e, right neighbour; mean edge
// lengths) assembled and restricted to the N+3 points (homogeneous Dirichlet
// just beyond the overlap); points outside the domain and Dirichlet boundary
// points decoupled.  A_e = Bz(x)By(x)Ax + Bz(x)Ay(x)Bx + Az(x)By(x)Bx is inverted
// by fast diagonalisation, A S = B S Lambda with S^T B S = I:
//   A_e^{-1} = (Sz(x)Sy(x)Sx) diag(1/(lz + ly + lx)) (Sz(x)Sy(x)Sx)^T.
// Coarse level: the trilinear (N = 1) mesh on the same vertices; P^T sums
// r/mult into the vertices, P interpolates back; A_c^{-1} by a fixed number
// of Jacobi-CG iterations (device-driven).
//
// GB300 design (FP32, the inner solver's precision): the 1-D eigenproblems
// are solved once on the host (Cholesky + cyclic Jacobi) and cached by their
// key (lengths and boundary flags: a tensor-product mesh has few distinct
// ones).  One warp per element, each lane owning whole 1-D lines: the K
// forward pass reads the extended residual straight from global memory
// (neighbour offsets computed from the box topology) and also restricts it
// to the element vertices; the J and I passes run through a padded shared
// block whose lines are dealt to the lanes by per-pass tables that avoid
// bank conflicts (the I pass does forward, division and backward in
// registers); the K backward pass stores straight to global memory.  Table
// rows are broadcast 16-byte loads and the multiply-adds packed FP32x2.  The
// coarse problem is assembled once into a 27-point stencil on the global
// vertex grid and solved by one cooperative kernel (Jacobi-CG, two grid
// barriers per iteration, the search direction double-buffered so the
// operator rebuilds it on the fly).  A last kernel, one thread per (i, j)
// column of an element, sums each point's value over the (up to 2 x 2 x 2)
// overlapping subdomains in a fixed order and adds the trilinear
// prolongation of the coarse solution: deterministic, copies of a node
// bit-identical, no atomics.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "sem_common.cuh"

struct sem_schwarz {
    const sem_mesh *m, *mc;
    int N, ne, P;
    int nv;        // coarse (global vertex) unknowns
    float *S;      // [P][ne][ne] eigenvectors S[l][a] (row l = point, column a = mode)
    float *L;      // [P][ne] eigenvalues
    int *prob;     // [E][3] problem id per element and axis
    float *uext;   // [E][ne^3] extended local solutions
    float *rce;    // [E][8] element restrictions of r / mult to the vertices
    float *sten;   // [27][nv] assembled coarse operator, offset (ox,oy,oz) -> (ox+1) + 3(oy+1) + 9(oz+1)
    float *cdinv;  // [nv] inverse coarse diagonal (0 on Dirichlet vertices)
    float *xc, *rcg, *pc0, *pc1, *wc;  // [nv] coarse CG vectors
    double *partial;  // [2][kCgMaxGrid]
    unsigned *bar;    // grid barrier counter
    float *J1;        // [2][kMaxN1] J1[a][i] = (1 -+ xi_i) / 2
    short *lines;     // [3][32 LPT] line dealt to each (group, lane) slot of a pass, or -1
    size_t ws_bytes;
};

namespace sem {

// ---------------------------------------------------------------- host set-up

// Generalised symmetric eigenproblem A s = lambda B s (B SPD): Cholesky B =
// G G^T, C = G^-1 A G^-T, cyclic Jacobi rotations C = V diag(l) V^T,
// S = G^-T V (so S^T B S = I, S^T A S = diag(l)).
static void gen_eig(int n, const double *A, const double *B, double *S, double *lam) {
    std::vector<double> G(n * n, 0.0), C(n * n), V(n * n, 0.0), T(n * n);
    for (int j = 0; j < n; ++j) {
        double d = B[j * n + j];
        for (int k = 0; k < j; ++k) d -= G[j * n + k] * G[j * n + k];
        G[j * n + j] = std::sqrt(d);
        for (int i = j + 1; i < n; ++i) {
            double v = B[i * n + j];
            for (int k = 0; k < j; ++k) v -= G[i * n + k] * G[j * n + k];
            G[i * n + j] = v / G[j * n + j];
        }
    }
    // T = G^-1 A (forward substitution per column), C = T G^-T (per row)
    for (int c = 0; c < n; ++c)
        for (int i = 0; i < n; ++i) {
            double v = A[i * n + c];
            for (int k = 0; k < i; ++k) v -= G[i * n + k] * T[k * n + c];
            T[i * n + c] = v / G[i * n + i];
        }
    for (int r = 0; r < n; ++r)
        for (int j = 0; j < n; ++j) {
            double v = T[r * n + j];
            for (int k = 0; k < j; ++k) v -= C[r * n + k] * G[j * n + k];
            C[r * n + j] = v / G[j * n + j];
        }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) C[i * n + j] = C[j * n + i] = 0.5 * (C[i * n + j] + C[j * n + i]);
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += C[i * n + j] * C[i * n + j];
                if (i != j) off += C[i * n + j] * C[i * n + j];
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = C[p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double theta = (C[q * n + q] - C[p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double ckp = C[k * n + p], ckq = C[k * n + q];
                    C[k * n + p] = c * ckp - s * ckq;
                    C[k * n + q] = s * ckp + c * ckq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double cpk = C[p * n + k], cqk = C[q * n + k];
                    C[p * n + k] = c * cpk - s * cqk;
                    C[q * n + k] = s * cpk + c * cqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) lam[i] = C[i * n + i];
    // S = G^-T V: back substitution per column
    for (int c = 0; c < n; ++c)
        for (int i = n - 1; i >= 0; --i) {
            double v = V[i * n + c];
            for (int k = i + 1; k < n; ++k) v -= G[k * n + i] * S[k * n + c];
            S[i * n + c] = v / G[i * n + i];
        }
}

// Cache key of a 1-D problem: lengths on a log scale with 2^-10 relative
// resolution (exact repeats on tensor-product meshes; nearby ones merged on
// deformed meshes, a change far below what matters to a preconditioner) and
// the boundary flags.
struct FdmKey {
    long long h, hL, hR;
    int flags;
    bool operator<(const FdmKey &o) const {
        if (flags != o.flags) return flags < o.flags;
        if (h != o.h) return h < o.h;
        if (hL != o.hL) return hL < o.hL;
        return hR < o.hR;
    }
};
static long long qlen(double h) { return std::llround(std::log2(h) * 1024.0); }

// Reference 1-D stiffness Ah[i][j] = sum_q D_qi rho_q D_qj and mass weights
// Bh[i] = rho_i on [-1, 1].
static void ref_1d(int N, const double *rho, const double *D, double *Ah, double *Bh) {
    const int n1 = N + 1;
    for (int i = 0; i < n1; ++i) {
        Bh[i] = rho[i];
        for (int j = 0; j < n1; ++j) {
            double s = 0.0;
            for (int q = 0; q < n1; ++q) s += D[q * n1 + i] * rho[q] * D[q * n1 + j];
            Ah[i * n1 + j] = s;
        }
    }
}

// The 1-D problem of an extended element along one axis (N + 3 points):
// stiffness and mass of the left neighbour, the element and the right
// neighbour (lengths hL, h, hR) assembled on 3N + 1 points and restricted to
// the N + 3 extended ones; a point without a neighbour (hasL / hasR false)
// and a Dirichlet boundary point (dirL / dirR) decoupled as identity rows;
// then A S = B S Lambda by gen_eig.
static void fdm_1d(int N, const double *Ah, const double *Bh, double h, double hL, double hR, bool hasL, bool hasR,
                   bool dirL, bool dirR, double *S, double *lam) {
    const int n1 = N + 1, ne = N + 3, M3 = 3 * N + 1;
    std::vector<double> Af(M3 * M3, 0.0), Bf(M3 * M3, 0.0), A(ne * ne), B(ne * ne);
    const double hh[3] = {hL, h, hR};
    for (int q = 0; q < 3; ++q)
        for (int i = 0; i < n1; ++i) {
            const int gi = q * N + i;
            Bf[gi * M3 + gi] += 0.5 * hh[q] * Bh[i];
            for (int j = 0; j < n1; ++j) Af[gi * M3 + q * N + j] += (2.0 / hh[q]) * Ah[i * n1 + j];
        }
    for (int i = 0; i < ne; ++i)
        for (int j = 0; j < ne; ++j) {
            A[i * ne + j] = Af[(N - 1 + i) * M3 + (N - 1 + j)];
            B[i * ne + j] = Bf[(N - 1 + i) * M3 + (N - 1 + j)];
        }
    const int dead[4] = {!hasL ? 0 : -1, dirL ? 1 : -1, !hasR ? ne - 1 : -1, dirR ? ne - 2 : -1};
    for (int d : dead) {
        if (d < 0) continue;
        for (int q = 0; q < ne; ++q) {
            A[d * ne + q] = A[q * ne + d] = 0.0;
            B[d * ne + q] = B[q * ne + d] = 0.0;
        }
        A[d * ne + d] = B[d * ne + d] = 1.0;
    }
    gen_eig(ne, A.data(), B.data(), S, lam);
}

// ---------------------------------------------------------------- kernels

constexpr int kSwWarps = 4;       // elements (one per warp) per CTA of the local solve
constexpr int kCgThreads = 256;   // coarse CG CTA (256 measured faster than 512 and 1024)
constexpr int kCgMaxGrid = 1024;  // coarse CG CTAs at most (one per SM)

struct SwArgs {
    int E;
    int nel[3], per[3], faces;
};

// Global vertex grid of the box: nv[a] = nel[a] (periodic) or nel[a] + 1.
struct CoarseTopo {
    int nel[3], per[3], nv[3], faces;
    int nvt;
};

// Extended-block geometry of order N: NE = N + 3 points per direction, LPT
// lines per lane (NE^2 lines over 32 lanes), table rows padded to NEP, block
// strides PJ (J) and PK (K) in floats.  Within a pass all of a lane's
// accesses move by the same stride, so a group of 32 lines (one per lane) is
// conflict-free when its start addresses fall in distinct banks: the strides
// are chosen (exhaustive search) so that at most LPT line starts share a bank
// in every direction where that is possible with little padding (N = 3, 4,
// 6, 7), and the lines are dealt to the lanes by a per-pass table (see
// line_table) that keeps equal banks in different groups.
template <int N>
struct SwShape {
    static constexpr int N1 = N + 1, NPT = N1 * N1 * N1;
    static constexpr int NE = N + 3, NE2 = NE * NE, NE3 = NE2 * NE;
    static constexpr int LPT = (NE2 + 31) / 32;
    static constexpr int NEP = (NE + 3) / 4 * 4;
    static constexpr int PJ = N == 5 ? 9 : N == 9 ? 13 : NE;
    static constexpr int PK = N == 2   ? 25
                              : N == 3 ? 37
                              : N == 4 ? 52
                              : N == 5 ? 72
                              : N == 6 ? 93
                              : N == 7 ? 103
                              : N == 8 ? 121
                                       : 156;
    static constexpr int SLOTS = 32 * LPT;  // line slots of a pass (line id or -1)
    static constexpr int TAB = 3 * NE * NEP;                 // one table set (3 axes)
    static constexpr int LAM = (3 * NE + 3) / 4 * 4;
    static constexpr int BUF = (PK * NE + 3) / 4 * 4;
    static constexpr int OFF = (6 * NE + 3) / 4 * 4;           // 3 NE source offsets (int64)
    static constexpr int WARP_FLOATS = 2 * TAB + LAM + BUF + OFF;  // per warp: S rows, S^T rows, eigenvalues, block, offsets
    static_assert(PJ >= NE && PK >= PJ * NE, "block strides");
};

// Along one axis: the (element-coordinate offset, local index) of extended
// point I of an element at coordinate c of n (false outside the domain).
__device__ __forceinline__ bool ext_move(int I, int N, int c, int n, int per, int &dc, int &li) {
    if (I == 0) {
        if (c == 0 && !per) return false;
        dc = c == 0 ? n - 1 : -1;
        li = N - 1;
    } else if (I == N + 2) {
        if (c == n - 1 && !per) return false;
        dc = c == n - 1 ? -(n - 1) : 1;
        li = 1;
    } else {
        dc = 0;
        li = I - 1;
    }
    return true;
}

// 1/mult factor along one axis of local index i: 1/2 on a face shared with a
// neighbour (or with itself across a periodic direction of one element).
__device__ __forceinline__ float mult_fac(int i, int N, int c, int n, int per) {
    return ((i == 0 && (c > 0 || per)) || (i == N && (c < n - 1 || per))) ? 0.5f : 1.f;
}

__device__ __forceinline__ float f4c(const float4 &v, int c) {
    return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w;
}
__device__ __forceinline__ float2 f4p(const float4 &v, int h) {
    return h == 0 ? make_float2(v.x, v.y) : make_float2(v.z, v.w);
}

// acc[q][.] += row (NE entries, rw) * x[q] for the lane's LPT lines, outputs
// in packed pairs (FP32x2 multiply-adds; a scalar tail when NE is odd).
template <int NE, int NEP, int LPT>
__device__ __forceinline__ void row_fma(float2 (&acc)[LPT][NE / 2], float (&tail)[LPT], const float4 (&rw)[NEP / 4],
                                        const float (&x)[LPT]) {
#pragma unroll
    for (int q = 0; q < LPT; ++q) {
        const float2 xx = make_float2(x[q], x[q]);
#pragma unroll
        for (int a2 = 0; a2 < NE / 2; ++a2) acc[q][a2] = __ffma2_rn(f4p(rw[a2 / 2], a2 & 1), xx, acc[q][a2]);
        if (NE & 1) tail[q] = fmaf(f4c(rw[(NE - 1) / 4], (NE - 1) & 3), x[q], tail[q]);
    }
}

template <int NE, int LPT>
__device__ __forceinline__ float acc_at(const float2 (&acc)[LPT][NE / 2], const float (&tail)[LPT], int q, int a) {
    return (NE & 1) && a == NE - 1 ? tail[q] : ((a & 1) ? acc[q][a / 2].y : acc[q][a / 2].x);
}

// The lane's lines of the warp's block along axis AX from the pass's line
// table (line id c1 + NE c2, or -1): (c1, c2) = (J, K), (I, K) or (I, J);
// offsets into the block.
template <int N, int AX>
__device__ __forceinline__ void line_offsets(const short *lines, int lane, int (&off)[SwShape<N>::LPT],
                                             int (&c1)[SwShape<N>::LPT], int (&c2)[SwShape<N>::LPT],
                                             bool (&ok)[SwShape<N>::LPT]) {
    using S = SwShape<N>;
#pragma unroll
    for (int q = 0; q < S::LPT; ++q) {
        int id = lines[AX * S::SLOTS + 32 * q + lane];
        ok[q] = id >= 0;
        id = ok[q] ? id : 0;
        c1[q] = id % S::NE;
        c2[q] = id / S::NE;
        off[q] = AX == 0 ? S::PJ * c1[q] + S::PK * c2[q] : AX == 1 ? c1[q] + S::PK * c2[q] : c1[q] + S::PJ * c2[q];
    }
}

// One 1-D contraction of the warp's block along axis AX, each lane on its
// lines: out[a] = sum_l tab[AX][l][a] in[l] (in place), tab the S rows
// (forward: S^T along the line) or the S^T rows (backward: S).
template <int N, int AX>
__device__ __forceinline__ void sw_lines(float *buf, const float *tab, const short *lines, int lane) {
    using S = SwShape<N>;
    constexpr int NE = S::NE, LPT = S::LPT, NEP = S::NEP;
    constexpr int ST = AX == 0 ? 1 : AX == 1 ? S::PJ : S::PK;
    int off[LPT], c1[LPT], c2[LPT];
    bool ok[LPT];
    line_offsets<N, AX>(lines, lane, off, c1, c2, ok);
    float2 acc[LPT][NE / 2];
    float tail[LPT];
#pragma unroll
    for (int q = 0; q < LPT; ++q) {
        tail[q] = 0.f;
#pragma unroll
        for (int a2 = 0; a2 < NE / 2; ++a2) acc[q][a2] = make_float2(0.f, 0.f);
    }
    const float *t = tab + AX * NE * NEP;
#pragma unroll
    for (int l = 0; l < NE; ++l) {
        float x[LPT];
#pragma unroll
        for (int q = 0; q < LPT; ++q) x[q] = buf[off[q] + l * ST];
        float4 rw[NEP / 4];
#pragma unroll
        for (int c4 = 0; c4 < NEP / 4; ++c4) rw[c4] = reinterpret_cast<const float4 *>(t + l * NEP)[c4];
        row_fma<NE, NEP, LPT>(acc, tail, rw, x);
    }
#pragma unroll
    for (int q = 0; q < LPT; ++q)
        if (ok[q]) {
#pragma unroll
            for (int a = 0; a < NE; ++a) buf[off[q] + a * ST] = acc_at<NE, LPT>(acc, tail, q, a);
        }
}

// One direction done whole in registers: forward (S^T of axis AX), division
// by lambda_AX[a] + the lines' two other eigenvalues (the lines are indexed
// by modes then), backward (S).  Lines from the pass's line table.
template <int N, int AX>
__device__ __forceinline__ void sw_fused(float *buf, const float *tabS, const float *tabT, const float *lam,
                                         const short *lines, int lane) {
    using S = SwShape<N>;
    constexpr int NE = S::NE, LPT = S::LPT, NEP = S::NEP;
    constexpr int ST = AX == 0 ? 1 : AX == 1 ? S::PJ : S::PK;
    constexpr int L1 = AX == 0 ? 1 : 0, L2 = AX == 2 ? 1 : 2;  // axes of c1, c2
    int off[LPT], c1[LPT], c2[LPT];
    bool ok[LPT];
    line_offsets<N, AX>(lines, lane, off, c1, c2, ok);
    float2 acc[LPT][NE / 2];
    float tail[LPT];
#pragma unroll
    for (int q = 0; q < LPT; ++q) {
        tail[q] = 0.f;
#pragma unroll
        for (int a2 = 0; a2 < NE / 2; ++a2) acc[q][a2] = make_float2(0.f, 0.f);
    }
    const float *tS = tabS + AX * NE * NEP, *tT = tabT + AX * NE * NEP;
#pragma unroll
    for (int l = 0; l < NE; ++l) {
        float x[LPT];
#pragma unroll
        for (int q = 0; q < LPT; ++q) x[q] = buf[off[q] + l * ST];
        float4 rw[NEP / 4];
#pragma unroll
        for (int c4 = 0; c4 < NEP / 4; ++c4) rw[c4] = reinterpret_cast<const float4 *>(tS + l * NEP)[c4];
        row_fma<NE, NEP, LPT>(acc, tail, rw, x);
    }
    float lq[LPT];
#pragma unroll
    for (int q = 0; q < LPT; ++q) lq[q] = lam[L1 * NE + c1[q]] + lam[L2 * NE + c2[q]];
    float2 out[LPT][NE / 2];
    float otail[LPT];
#pragma unroll
    for (int q = 0; q < LPT; ++q) {
        otail[q] = 0.f;
#pragma unroll
        for (int a2 = 0; a2 < NE / 2; ++a2) out[q][a2] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int c = 0; c < NE; ++c) {
        const float la = lam[AX * NE + c];
        float x[LPT];
#pragma unroll
        for (int q = 0; q < LPT; ++q) x[q] = __fdividef(acc_at<NE, LPT>(acc, tail, q, c), lq[q] + la);
        float4 rw[NEP / 4];
#pragma unroll
        for (int c4 = 0; c4 < NEP / 4; ++c4) rw[c4] = reinterpret_cast<const float4 *>(tT + c * NEP)[c4];
        row_fma<NE, NEP, LPT>(out, otail, rw, x);
    }
#pragma unroll
    for (int q = 0; q < LPT; ++q)
        if (ok[q]) {
#pragma unroll
            for (int a = 0; a < NE; ++a) buf[off[q] + a * ST] = acc_at<NE, LPT>(out, otail, q, a);
        }
}

// Local solves: one warp per element.  uext[e] = A_e^{-1} R_e r on the
// extended points ([K][J][I], NE^3); with rce, also the restriction
// rce[e][a + 2b + 4c] = sum_ijk J1[a][i] J1[b][j] J1[c][k] r(i,j,k) / mult.
// Passes: K forward straight from global memory (lanes on (I, J) lines in
// natural order; the restriction from the same registers), J forward, I
// forward + division + I backward, J backward, K backward straight to
// global memory (for each K the warp stores 32 consecutive points).
// done (optional): a device flag; set -> return at once.
template <int N>
__global__ void __launch_bounds__(kSwWarps * 32, N <= 6 ? 5 : 4)
    schwarz_local_kernel(const float *__restrict__ r, const float *__restrict__ Stab, const float *__restrict__ Ltab,
                         const int *__restrict__ prob, const float *__restrict__ J1, const short *__restrict__ ltab,
                         SwArgs A, const int *__restrict__ done, float *__restrict__ uext,
                         float *__restrict__ rce) {
    using S = SwShape<N>;
    constexpr int NE = S::NE, NE2 = S::NE2, NE3 = S::NE3, N1 = S::N1, NPT = S::NPT, NEP = S::NEP, LPT = S::LPT;
    if (done && *done) return;
    extern __shared__ float4 sw_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *sS = reinterpret_cast<float *>(sw_smem) + warp * S::WARP_FLOATS;
    float *sT = sS + S::TAB, *sL = sT + S::TAB, *buf = sL + S::LAM;
    int64_t *sOff = reinterpret_cast<int64_t *>(buf + S::BUF);
    constexpr int64_t kOut = INT64_MIN;  // source outside the domain
    short *lines = reinterpret_cast<short *>(reinterpret_cast<float *>(sw_smem) + kSwWarps * S::WARP_FLOATS);
    for (int t = threadIdx.x; t < 3 * S::SLOTS; t += blockDim.x) lines[t] = ltab[t];
    __syncthreads();
    const int sy = A.nel[0], sz = A.nel[0] * A.nel[1];
    // the lane's K lines (I, J), natural order
    int kI[LPT], kJ[LPT];
    bool kok[LPT];
#pragma unroll
    for (int q = 0; q < LPT; ++q) {
        const int L = lane + 32 * q;
        kok[q] = L < NE2;
        kI[q] = kok[q] ? L % NE : 0;
        kJ[q] = kok[q] ? L / NE : 0;
    }
    for (int e = blockIdx.x * kSwWarps + warp; e < A.E; e += gridDim.x * kSwWarps) {
        __syncwarp();
        const int ex = e % A.nel[0], ey = (e / A.nel[0]) % A.nel[1], ez = e / sz;
        const int pid[3] = {__ldg(prob + 3 * (int64_t)e), __ldg(prob + 3 * (int64_t)e + 1),
                            __ldg(prob + 3 * (int64_t)e + 2)};
        constexpr int kTt = (3 * NE2 + 31) / 32;
        float tv[kTt];
#pragma unroll
        for (int u = 0; u < kTt; ++u) {
            const int t = lane + 32 * u;
            if (t < 3 * NE2) {
                const int a = t / NE2;
                tv[u] = __ldg(Stab + (int64_t)(a == 0 ? pid[0] : a == 1 ? pid[1] : pid[2]) * NE2 + (t - a * NE2));
            }
        }
        constexpr int kLt = (3 * NE + 31) / 32;
        float lv[kLt];
#pragma unroll
        for (int u = 0; u < kLt; ++u) {
            const int t = lane + 32 * u;
            if (t < 3 * NE) {
                const int a = t / NE;
                lv[u] = __ldg(Ltab + (int64_t)(a == 0 ? pid[0] : a == 1 ? pid[1] : pid[2]) * NE + (t - a * NE));
            }
        }
        // per axis, the offset of each extended point's source in r (element
        // offset x points per element + local stride), or kOut outside the domain
        for (int t = lane; t < 3 * NE; t += 32) {
            const int ax = t / NE, I = t - ax * NE;
            const int c = ax == 0 ? ex : ax == 1 ? ey : ez;
            const int n = ax == 0 ? A.nel[0] : ax == 1 ? A.nel[1] : A.nel[2];
            const int per = ax == 0 ? A.per[0] : ax == 1 ? A.per[1] : A.per[2];
            const int64_t es = ax == 0 ? 1 : ax == 1 ? sy : sz;
            const int ls = ax == 0 ? 1 : ax == 1 ? N1 : N1 * N1;
            int dc, li;
            sOff[t] = ext_move(I, N, c, n, per, dc, li) ? (dc * es) * NPT + (int64_t)li * ls : kOut;
        }
#pragma unroll
        for (int u = 0; u < kTt; ++u) {
            const int t = lane + 32 * u;
            if (t < 3 * NE2) {
                const int a = t / NE2, q = t - a * NE2, l = q / NE, c = q - l * NE;
                sS[(a * NE + l) * NEP + c] = tv[u];
                sT[(a * NE + c) * NEP + l] = tv[u];
            }
        }
#pragma unroll
        for (int u = 0; u < kLt; ++u)
            if (lane + 32 * u < 3 * NE) sL[lane + 32 * u] = lv[u];
        __syncwarp();
        // ---- K forward from global memory (+ restriction)
        {
            const float *re = r + (int64_t)e * NPT;
            int64_t oxy[LPT];
            bool vxy[LPT];
#pragma unroll
            for (int q = 0; q < LPT; ++q) {
                const int64_t ox = sOff[kI[q]], oy = sOff[NE + kJ[q]];
                vxy[q] = kok[q] && ox != kOut && oy != kOut;
                oxy[q] = vxy[q] ? ox + oy : 0;
            }
            float2 acc[LPT][NE / 2];
            float tail[LPT], rs0[LPT], rs1[LPT];
#pragma unroll
            for (int q = 0; q < LPT; ++q) {
                tail[q] = rs0[q] = rs1[q] = 0.f;
#pragma unroll
                for (int a2 = 0; a2 < NE / 2; ++a2) acc[q][a2] = make_float2(0.f, 0.f);
            }
            const float *tS = sS + 2 * NE * NEP;
#pragma unroll
            for (int K = 0; K < NE; ++K) {
                const int64_t oz = sOff[2 * NE + K];
                float x[LPT];
#pragma unroll
                for (int q = 0; q < LPT; ++q) x[q] = (vxy[q] && oz != kOut) ? __ldg(re + (oxy[q] + oz)) : 0.f;
                if (rce && K >= 1 && K <= N + 1) {
                    const float wz = mult_fac(K - 1, N, ez, A.nel[2], A.per[2]);
                    const float jz0 = __ldg(J1 + K - 1) * wz, jz1 = __ldg(J1 + kMaxN1 + K - 1) * wz;
#pragma unroll
                    for (int q = 0; q < LPT; ++q) {
                        rs0[q] = fmaf(jz0, x[q], rs0[q]);
                        rs1[q] = fmaf(jz1, x[q], rs1[q]);
                    }
                }
                float4 rw[NEP / 4];
#pragma unroll
                for (int c4 = 0; c4 < NEP / 4; ++c4) rw[c4] = reinterpret_cast<const float4 *>(tS + K * NEP)[c4];
                row_fma<NE, NEP, LPT>(acc, tail, rw, x);
            }
            if (rce) {
                float c8[8];
#pragma unroll
                for (int v = 0; v < 8; ++v) c8[v] = 0.f;
#pragma unroll
                for (int q = 0; q < LPT; ++q) {
                    const int i = kI[q] - 1, j = kJ[q] - 1;
                    if (kok[q] && i >= 0 && i <= N && j >= 0 && j <= N) {
                        const float wx = mult_fac(i, N, ex, A.nel[0], A.per[0]);
                        const float wy = mult_fac(j, N, ey, A.nel[1], A.per[1]);
                        const float x0 = __ldg(J1 + i) * wx, x1 = __ldg(J1 + kMaxN1 + i) * wx;
                        const float y0 = __ldg(J1 + j) * wy, y1 = __ldg(J1 + kMaxN1 + j) * wy;
                        c8[0] = fmaf(x0 * y0, rs0[q], c8[0]);
                        c8[1] = fmaf(x1 * y0, rs0[q], c8[1]);
                        c8[2] = fmaf(x0 * y1, rs0[q], c8[2]);
                        c8[3] = fmaf(x1 * y1, rs0[q], c8[3]);
                        c8[4] = fmaf(x0 * y0, rs1[q], c8[4]);
                        c8[5] = fmaf(x1 * y0, rs1[q], c8[5]);
                        c8[6] = fmaf(x0 * y1, rs1[q], c8[6]);
                        c8[7] = fmaf(x1 * y1, rs1[q], c8[7]);
                    }
                }
                float mine = 0.f;
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    float t = c8[v];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                    if (lane == v) mine = t;
                }
                if (lane < 8) rce[(int64_t)e * 8 + lane] = mine;
            }
#pragma unroll
            for (int q = 0; q < LPT; ++q)
                if (kok[q]) {
#pragma unroll
                    for (int c = 0; c < NE; ++c)
                        buf[kI[q] + S::PJ * kJ[q] + S::PK * c] = acc_at<NE, LPT>(acc, tail, q, c);
                }
        }
        __syncwarp();
        sw_lines<N, 1>(buf, sS, lines, lane);
        __syncwarp();
        sw_fused<N, 0>(buf, sS, sT, sL, lines, lane);
        __syncwarp();
        sw_lines<N, 1>(buf, sT, lines, lane);
        __syncwarp();
        // ---- K backward straight to global memory
        {
            float2 acc[LPT][NE / 2];
            float tail[LPT];
#pragma unroll
            for (int q = 0; q < LPT; ++q) {
                tail[q] = 0.f;
#pragma unroll
                for (int a2 = 0; a2 < NE / 2; ++a2) acc[q][a2] = make_float2(0.f, 0.f);
            }
            const float *tT = sT + 2 * NE * NEP;
#pragma unroll
            for (int c = 0; c < NE; ++c) {
                float x[LPT];
#pragma unroll
                for (int q = 0; q < LPT; ++q) x[q] = buf[kI[q] + S::PJ * kJ[q] + S::PK * c];
                float4 rw[NEP / 4];
#pragma unroll
                for (int c4 = 0; c4 < NEP / 4; ++c4) rw[c4] = reinterpret_cast<const float4 *>(tT + c * NEP)[c4];
                row_fma<NE, NEP, LPT>(acc, tail, rw, x);
            }
            float *ue = uext + (int64_t)e * NE3;
#pragma unroll
            for (int q = 0; q < LPT; ++q)
                if (kok[q]) {
#pragma unroll
                    for (int K = 0; K < NE; ++K) ue[K * NE2 + lane + 32 * q] = acc_at<NE, LPT>(acc, tail, q, K);
                }
        }
    }
}

// Along one axis: the subdomains covering local index i of an element at
// coordinate c of n, in three slots left to right: the left neighbour (its
// own point N, or its right extension), the element itself, the right
// neighbour (its own point 0, or its left extension); each with its
// element-coordinate offset and extended index.  (N = 2: the middle point is
// covered by all three.)
struct Cover {
    bool l, r;
    int dl, dr, Il, I0, Ir;
};
__device__ __forceinline__ Cover cover(int i, int N, int c, int n, int per) {
    Cover v;
    v.l = i <= 1 && (c > 0 || per);
    v.dl = c == 0 ? n - 1 : -1;
    v.Il = i + N + 1;
    v.I0 = i + 1;
    v.r = i >= N - 1 && (c < n - 1 || per);
    v.dr = c == n - 1 ? -(n - 1) : 1;
    v.Ir = i - N + 1;
    return v;
}
__device__ __forceinline__ bool cov_ok(const Cover &v, int slot) { return slot == 0 ? v.l : slot == 1 ? true : v.r; }
__device__ __forceinline__ int cov_d(const Cover &v, int slot) { return slot == 0 ? v.dl : slot == 1 ? 0 : v.dr; }
__device__ __forceinline__ int cov_I(const Cover &v, int slot) { return slot == 0 ? v.Il : slot == 1 ? v.I0 : v.Ir; }

__device__ __forceinline__ bool dirichlet_at(int i, int N, int c, int n, int per, int faces, int axis) {
    return !per && ((i == 0 && c == 0 && ((faces >> (2 * axis)) & 1)) ||
                    (i == N && c == n - 1 && ((faces >> (2 * axis + 1)) & 1)));
}

// Global vertex index of vertex (vx, vy, vz) in [0, nel] (periodic: nel wraps to 0).
__device__ __forceinline__ int vertex_id(const CoarseTopo &C, int vx, int vy, int vz) {
    if (C.per[0] && vx == C.nel[0]) vx = 0;
    if (C.per[1] && vy == C.nel[1]) vy = 0;
    if (C.per[2] && vz == C.nel[2]) vz = 0;
    return vx + C.nv[0] * (vy + C.nv[1] * vz);
}

// z(e, i, j, k) = sum over the covering subdomains (z, then y, then x from
// low to high position) of their extended solutions, plus (xc non-NULL) the
// trilinear interpolation of the coarse solution (x, then y, then z: exact at
// element faces, so copies stay identical); 0 on Dirichlet nodes.  One thread
// per (i, j) column of an element, k unrolled: the x/y covers, their offsets
// and the x/y interpolation are formed once per column.
template <int N>
constexpr int sum_epb() {  // elements per 256-thread CTA
    return 256 / ((N + 1) * (N + 1));
}

// Off: the type of the x/y neighbour offsets (int where nel_x nel_y (N+3)^3
// < 2^31, which halves their registers; int64_t otherwise).
template <int N, typename Off>
__global__ void __launch_bounds__(256, 4)
    schwarz_sum_kernel(const float *__restrict__ uext, const float *__restrict__ xc, const float *__restrict__ J1,
                       SwArgs A, CoarseTopo C, const int *__restrict__ done, float *__restrict__ z) {
    constexpr int N1 = N + 1, NE = N + 3, NE3 = NE * NE * NE, NPT = N1 * N1 * N1, COLS = N1 * N1;
    constexpr int EPB = sum_epb<N>();
    if (done && *done) return;
    __shared__ float sx[EPB][8];
    const int sy = A.nel[0], sz = A.nel[0] * A.nel[1];
    const int el = threadIdx.x / COLS, col = threadIdx.x - el * COLS;
    const int i = col % N1, j = col / N1;
    for (int e0 = blockIdx.x * EPB; e0 < A.E; e0 += gridDim.x * EPB) {
        const int e = e0 + el;
        const bool live = el < EPB && e < A.E;
        const int ex = e % A.nel[0], ey = (e / A.nel[0]) % A.nel[1], ez = e / sz;
        if (xc) {
            __syncthreads();
            if (live && col < 8)
                sx[el][col] = __ldcg(xc + vertex_id(C, ex + (col & 1), ey + ((col >> 1) & 1), ez + (col >> 2)));
            __syncthreads();
        }
        if (!live) continue;
        const bool dxy = dirichlet_at(i, N, ex, A.nel[0], A.per[0], A.faces, 0) ||
                         dirichlet_at(j, N, ey, A.nel[1], A.per[1], A.faces, 1);
        const Cover cx = cover(i, N, ex, A.nel[0], A.per[0]);
        const Cover cy = cover(j, N, ey, A.nel[1], A.per[1]);
        // x/y slot pairs (b outer, a inner): validity and offset
        bool okxy[9];
        Off oxy[9];
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                okxy[3 * b + a] = cov_ok(cy, b) && cov_ok(cx, a);
                oxy[3 * b + a] = (Off)(cov_d(cx, a) + sy * cov_d(cy, b)) * NE3 + cov_I(cx, a) + NE * cov_I(cy, b);
            }
        float u0 = 0.f, u1 = 0.f;
        if (xc) {
            const float jx0 = __ldg(J1 + i), jx1 = __ldg(J1 + kMaxN1 + i);
            const float jy0 = __ldg(J1 + j), jy1 = __ldg(J1 + kMaxN1 + j);
            const float *v = sx[el];
            const float t00 = fmaf(jx0, v[0], jx1 * v[1]), t10 = fmaf(jx0, v[2], jx1 * v[3]);
            const float t01 = fmaf(jx0, v[4], jx1 * v[5]), t11 = fmaf(jx0, v[6], jx1 * v[7]);
            u0 = fmaf(jy0, t00, jy1 * t10);
            u1 = fmaf(jy0, t01, jy1 * t11);
        }
        const float *ue = uext + (int64_t)e * NE3;
        float *ze = z + (int64_t)e * NPT + col;
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            const Cover cz = cover(k, N, ez, A.nel[2], A.per[2]);
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (cov_ok(cz, c)) {
                    const int64_t oz = (int64_t)(sz * cov_d(cz, c)) * NE3 + NE * NE * cov_I(cz, c);
#pragma unroll
                    for (int q = 0; q < 9; ++q)
                        if (okxy[q]) s += __ldg(ue + oz + oxy[q]);
                }
            if (xc) s += fmaf(__ldg(J1 + k), u0, __ldg(J1 + kMaxN1 + k) * u1);
            const bool dz = dirichlet_at(k, N, ez, A.nel[2], A.per[2], A.faces, 2);
            ze[k * COLS] = (dxy || dz) ? 0.f : s;
        }
    }
}

// ---------------------------------------------------------------- coarse level

// Element matrices of the N = 1 operator from its FP64 geometric factors
// G[e][6][8] (rr, ss, tt, rs, rt, st at the 8 vertices, quadrature weights
// included): Ae[e][p][j] = sum_q grad phi_p(q) . G(q) grad phi_j(q), with
// d phi_j / dr at vertex q = +-1/2 where q agrees with j off that axis.
// Column j of one element (Ge: its 48 factors, Ae_e: its 64 entries).  Host
// and device: the set-up kernel and the host query run this same code.
__host__ __device__ __forceinline__ void coarse_elem_col(const double *Ge, int j, float *Ae_e) {
    double col[8] = {};
    for (int q = 0; q < 8; ++q) {
        double gj[3];
        for (int a = 0; a < 3; ++a) {
            const int mask = 7 & ~(1 << a);
            gj[a] = ((q ^ j) & mask) ? 0.0 : (((j >> a) & 1) ? 0.5 : -0.5);
        }
        const double grr = Ge[q], gss = Ge[8 + q], gtt = Ge[16 + q], grs = Ge[24 + q], grt = Ge[32 + q],
                     gst = Ge[40 + q];
        const double v0 = grr * gj[0] + grs * gj[1] + grt * gj[2];
        const double v1 = grs * gj[0] + gss * gj[1] + gst * gj[2];
        const double v2 = grt * gj[0] + gst * gj[1] + gtt * gj[2];
        for (int p = 0; p < 8; ++p) {
            double gp[3];
            for (int a = 0; a < 3; ++a) {
                const int mask = 7 & ~(1 << a);
                gp[a] = ((q ^ p) & mask) ? 0.0 : (((p >> a) & 1) ? 0.5 : -0.5);
            }
            col[p] += gp[0] * v0 + gp[1] * v1 + gp[2] * v2;
        }
    }
    for (int p = 0; p < 8; ++p) Ae_e[p * 8 + j] = (float)col[p];
}

__global__ void coarse_elem_kernel(const double *__restrict__ G, int E, float *__restrict__ Ae) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)E * 8;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = t / 8;
        coarse_elem_col(G + e * 48, (int)(t - e * 8), Ae + e * 64);
    }
}

__host__ __device__ __forceinline__ bool vertex_masked(const CoarseTopo &C, int v, int a) {
    return !C.per[a] && ((v == 0 && ((C.faces >> (2 * a)) & 1)) || (v == C.nv[a] - 1 && ((C.faces >> (2 * a + 1)) & 1)));
}

// Neighbour coordinate v + o along an axis (periodic wrap); -1 outside.
__host__ __device__ __forceinline__ int nb_coord(int v, int o, int nv, int per) {
    int w = v + o;
    if (per) w = (w + nv) % nv;
    return (w < 0 || w >= nv) ? -1 : w;
}

// Element coordinate of the element holding vertex coordinate v at local
// vertex s (0 or 1); -1 if none.
__host__ __device__ __forceinline__ int elem_coord(int v, int s, int nel, int per) {
    int c = v - s;
    if (per) c = (c + nel) % nel;
    return (c < 0 || c >= nel) ? -1 : c;
}

// The assembled coarse operator as a 27-point stencil per vertex:
// sten[o][v] = sum over the (up to 8) elements e holding v at local vertex s
// (s in a fixed order) of Ae[e][s][s + o] for s + o in {0,1}^3 (periodic
// aliases included); rows and columns of Dirichlet vertices zeroed; cdinv the
// inverse of the assembled diagonal (0 on Dirichlet vertices).  One vertex;
// host and device.
__host__ __device__ __forceinline__ void coarse_stencil_row(const float *Ae, const CoarseTopo &C, int v, float *sten,
                                                            float *cdinv) {
    const int vc[3] = {v % C.nv[0], (v / C.nv[0]) % C.nv[1], v / (C.nv[0] * C.nv[1])};
    const bool mv = vertex_masked(C, vc[0], 0) || vertex_masked(C, vc[1], 1) || vertex_masked(C, vc[2], 2);
    double diag = 0.0;
    for (int o = 0; o < 27; ++o) {
        const int od[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
        int nc[3];
        bool ok = true, mn = false;
        for (int a = 0; a < 3; ++a) {
            nc[a] = nb_coord(vc[a], od[a], C.nv[a], C.per[a]);
            ok = ok && nc[a] >= 0;
        }
        double sum = 0.0;
        if (ok) {
            for (int a = 0; a < 3; ++a) mn = mn || vertex_masked(C, nc[a], a);
            for (int s = 0; s < 8; ++s) {
                const int sd[3] = {s & 1, (s >> 1) & 1, s >> 2};
                int ec[3], td = 0;
                bool in = true;
                for (int a = 0; a < 3; ++a) {
                    ec[a] = elem_coord(vc[a], sd[a], C.nel[a], C.per[a]);
                    const int ta = sd[a] + od[a];
                    in = in && ec[a] >= 0 && ta >= 0 && ta <= 1;
                    td |= (ta & 1) << a;
                }
                if (!in) continue;
                const int64_t e = ec[0] + (int64_t)C.nel[0] * (ec[1] + (int64_t)C.nel[1] * ec[2]);
                sum += Ae[e * 64 + s * 8 + td];
            }
            const int nbv = nc[0] + C.nv[0] * (nc[1] + C.nv[1] * nc[2]);
            if (nbv == v) diag += sum;
        }
        sten[(int64_t)o * C.nvt + v] = (ok && !mv && !mn) ? (float)sum : 0.f;
    }
    cdinv[v] = (mv || !(diag > 0.0)) ? 0.f : (float)(1.0 / diag);
}

__global__ void coarse_stencil_kernel(const float *__restrict__ Ae, CoarseTopo C, float *__restrict__ sten,
                                      float *__restrict__ cdinv) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < C.nvt; v += gridDim.x * blockDim.x)
        coarse_stencil_row(Ae, C, v, sten, cdinv);
}

struct CoarseArgs {
    const float *sten, *cdinv, *rce;
    float *x, *r, *p0, *p1, *w;
    double *partial;  // [2][kCgMaxGrid]
    unsigned *bar;
    int *err;
    const int *done;
    CoarseTopo C;
    int iters;
    double tol2;
};

// Block sum of v into partial[blockIdx.x]; after the barrier every CTA sums
// the partials in the same fixed order (identical totals everywhere).
__device__ __forceinline__ void cg_block_partial(double v, double *partial) {
    __shared__ double sh[kCgThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kCgThreads / 32; ++k) t += sh[k];
        __stcg(partial + blockIdx.x, t);
    }
}

__device__ __forceinline__ double cg_total(const double *partial) {
    __shared__ double tot;
    if (threadIdx.x < 32) {
        double t = 0.0;
        for (int k = threadIdx.x; k < (int)gridDim.x; k += 32) t += __ldcg(partial + k);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) tot = t;
    }
    __syncthreads();
    const double v = tot;
    __syncthreads();
    return v;
}

// Per-vertex steps of the coarse CG, shared by the cooperative kernel and
// the multi-kernel form.
// Right-hand side of vertex v: the sum over the elements holding v (fixed
// order) of their restrictions, 0 on Dirichlet vertices; also r = b,
// x = p_old = 0.  Returns b (D^-1 b b of the first rz).
__device__ __forceinline__ float coarse_rhs_vertex(const CoarseArgs &P, int v) {
    const CoarseTopo &C = P.C;
    const int vx = v % C.nv[0], vy = (v / C.nv[0]) % C.nv[1], vz = v / (C.nv[0] * C.nv[1]);
    float b = 0.f;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const int ex = elem_coord(vx, s & 1, C.nel[0], C.per[0]);
        const int ey = elem_coord(vy, (s >> 1) & 1, C.nel[1], C.per[1]);
        const int ez = elem_coord(vz, s >> 2, C.nel[2], C.per[2]);
        if (ex < 0 || ey < 0 || ez < 0) continue;
        b += __ldg(P.rce + (ex + (int64_t)C.nel[0] * (ey + (int64_t)C.nel[1] * ez)) * 8 + s);
    }
    if (__ldg(P.cdinv + v) == 0.f) b = 0.f;
    __stcg(P.r + v, b);
    __stcg(P.x + v, 0.f);
    __stcg(P.p0 + v, 0.f);
    return b;
}

// p_new(v) = cdinv r + beta p_old at v and w(v) = (A_c p_new)(v), the
// neighbours' p_new rebuilt from their r and p_old.  Returns p_new(v).
__device__ __forceinline__ float coarse_apply_vertex(const CoarseArgs &P, int v, float beta, const float *pold,
                                                     float &w) {
    const CoarseTopo &C = P.C;
    const int nvt = C.nvt;
    const int vx = v % C.nv[0], vy = (v / C.nv[0]) % C.nv[1], vz = v / (C.nv[0] * C.nv[1]);
    int nx[3], ny[3], nz[3];
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        nx[o] = nb_coord(vx, o - 1, C.nv[0], C.per[0]);
        ny[o] = nb_coord(vy, o - 1, C.nv[1], C.per[1]);
        nz[o] = nb_coord(vz, o - 1, C.nv[2], C.per[2]);
    }
    float acc = 0.f;
#pragma unroll
    for (int o = 0; o < 27; ++o) {
        const int a = nx[o % 3], b = ny[(o / 3) % 3], c = nz[o / 9];
        if (a < 0 || b < 0 || c < 0) continue;
        const int q = a + C.nv[0] * (b + C.nv[1] * c);
        const float pq = fmaf(beta, __ldcg(pold + q), __ldg(P.cdinv + q) * __ldcg(P.r + q));
        acc = fmaf(__ldg(P.sten + (int64_t)o * nvt + v), pq, acc);
    }
    w = acc;
    return fmaf(beta, __ldcg(pold + v), __ldg(P.cdinv + v) * __ldcg(P.r + v));
}

// The coarse solve A_c x = b, b assembled from the element restrictions,
// x0 = 0, up to `iters` Jacobi-CG iterations or rz <= tol2 rz0.  Per
// iteration: (1) p_new = cdinv r + beta p_old for the owned vertices and
// w = A_c p_new, the neighbours' p_new rebuilt from their r and p_old (no
// barrier between the two), <p, w>; (2) x, r update, <r, cdinv r>.  Two grid
// barriers per iteration.  Cooperative launch, grid <= one CTA per SM.
__global__ void __launch_bounds__(kCgThreads) coarse_cg_kernel(CoarseArgs P) {
    if (P.done && *P.done) return;
    const CoarseTopo &C = P.C;
    const int nvt = C.nvt;
    const int stride = gridDim.x * blockDim.x;
    unsigned nbar = 0;
    // b = sum over the elements holding v (fixed order) of their restriction
    double part = 0.0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nvt; v += stride) {
        const float b = coarse_rhs_vertex(P, v);
        part += (double)b * (double)(__ldg(P.cdinv + v) * b);
    }
    cg_block_partial(part, P.partial);
    if (!grid_barrier_bounded(P.bar, ++nbar * gridDim.x, P.err)) return;
    double rz = cg_total(P.partial);
    const double rz0 = rz;
    float beta = 0.f;
    float *pold = P.p0, *pnew = P.p1;
    for (int it = 0; it < P.iters; ++it) {
        if (!(rz > P.tol2 * rz0)) break;
        part = 0.0;
        for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nvt; v += stride) {
            float w;
            const float pv = coarse_apply_vertex(P, v, beta, pold, w);
            __stcg(pnew + v, pv);
            __stcg(P.w + v, w);
            part += (double)pv * (double)w;
        }
        cg_block_partial(part, P.partial);
        if (!grid_barrier_bounded(P.bar, ++nbar * gridDim.x, P.err)) return;
        const double pw = cg_total(P.partial);
        const float alpha = pw != 0.0 ? (float)(rz / pw) : 0.f;
        part = 0.0;
        for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nvt; v += stride) {
            const float pv = __ldcg(pnew + v), wv = __ldcg(P.w + v);
            __stcg(P.x + v, fmaf(alpha, pv, __ldcg(P.x + v)));
            const float rv = fmaf(-alpha, wv, __ldcg(P.r + v));
            __stcg(P.r + v, rv);
            part += (double)rv * (double)(__ldg(P.cdinv + v) * rv);
        }
        cg_block_partial(part, P.partial + kCgMaxGrid);
        if (!grid_barrier_bounded(P.bar, ++nbar * gridDim.x, P.err)) return;
        const double rzn = cg_total(P.partial + kCgMaxGrid);
        beta = rz != 0.0 ? (float)(rzn / rz) : 0.f;
        rz = rzn;
        float *t = pold;
        pold = pnew;
        pnew = t;
    }
}

// ---- the coarse CG as separate launches (no grid barrier)
//
// The same iteration in three kernels -- right-hand side and rz0, then per
// iteration p_new and A_c p_new with <p, A_c p>, then the x and r updates
// with <r, D^-1 r> -- each closed by a deterministic last-block reduction
// (block partials, summed in block order by the last block to arrive).  For
// graphs whose branches run concurrently: a cooperative grid must not wait
// on CTAs that other branches' kernels keep from being scheduled.  An early
// stop (rz <= tol2 rz0) turns the remaining launches into no-ops.
struct CoarseScal {
    unsigned bar;   // grid barrier counter of the cooperative form
    unsigned cnt;   // arrival counter of the last-block reductions
    int stop;       // 1: the iteration is over
    int pad;
    double rz, rz0, pw;
    float alpha, beta;
};

// Block partial of v; in the last block to arrive, tot = the sum of all
// partials in block order (every thread) and the counter is reset.
__device__ __forceinline__ bool coarse_last_block(double v, double *partial, unsigned *cnt, double &tot) {
    __shared__ int last;
    cg_block_partial(v, partial);
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(cnt, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    tot = cg_total(partial);
    if (threadIdx.x == 0) *cnt = 0u;
    return true;
}

__global__ void __launch_bounds__(kCgThreads) coarse_mk_init_kernel(CoarseArgs P, CoarseScal *S) {
    if (P.done && *P.done) return;
    double part = 0.0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < P.C.nvt; v += gridDim.x * blockDim.x) {
        const float b = coarse_rhs_vertex(P, v);
        part += (double)b * (double)(__ldg(P.cdinv + v) * b);
    }
    double tot;
    if (coarse_last_block(part, P.partial, &S->cnt, tot) && threadIdx.x == 0) {
        S->rz = tot;
        S->rz0 = tot;
        S->beta = 0.f;
        S->stop = (P.iters > 0 && tot > P.tol2 * tot) ? 0 : 1;
    }
}

__global__ void __launch_bounds__(kCgThreads)
    coarse_mk_pw_kernel(CoarseArgs P, CoarseScal *S, const float *pold, float *pnew) {
    if ((P.done && *P.done) || S->stop) return;
    const float beta = S->beta;
    double part = 0.0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < P.C.nvt; v += gridDim.x * blockDim.x) {
        float w;
        const float pv = coarse_apply_vertex(P, v, beta, pold, w);
        __stcg(pnew + v, pv);
        __stcg(P.w + v, w);
        part += (double)pv * (double)w;
    }
    double tot;
    if (coarse_last_block(part, P.partial, &S->cnt, tot) && threadIdx.x == 0) {
        S->pw = tot;
        S->alpha = tot != 0.0 ? (float)(S->rz / tot) : 0.f;
    }
}

__global__ void __launch_bounds__(kCgThreads) coarse_mk_xr_kernel(CoarseArgs P, CoarseScal *S, const float *pnew) {
    if ((P.done && *P.done) || S->stop) return;
    const float alpha = S->alpha;
    double part = 0.0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < P.C.nvt; v += gridDim.x * blockDim.x) {
        const float pv = __ldcg(pnew + v), wv = __ldcg(P.w + v);
        __stcg(P.x + v, fmaf(alpha, pv, __ldcg(P.x + v)));
        const float rv = fmaf(-alpha, wv, __ldcg(P.r + v));
        __stcg(P.r + v, rv);
        part += (double)rv * (double)(__ldg(P.cdinv + v) * rv);
    }
    double tot;
    if (coarse_last_block(part, P.partial + kCgMaxGrid, &S->cnt, tot) && threadIdx.x == 0) {
        const double rz = S->rz;
        S->beta = rz != 0.0 ? (float)(tot / rz) : 0.f;
        S->rz = tot;
        S->stop = tot > P.tol2 * S->rz0 ? 0 : 1;
    }
}

// ---------------------------------------------------------------- host side

static CoarseTopo coarse_topo(const int *nel, const int *periodic, int faces) {
    CoarseTopo C;
    C.nvt = 1;
    for (int a = 0; a < 3; ++a) {
        C.nel[a] = nel[a];
        C.per[a] = periodic[a] ? 1 : 0;
        C.nv[a] = nel[a] + (periodic[a] ? 0 : 1);
        C.nvt *= C.nv[a];
    }
    C.faces = faces;
    return C;
}

static CoarseTopo coarse_topo(const sem_mesh *m) { return coarse_topo(m->nel, m->periodic, m->faces); }

// Deal the NE^2 lines of the I and J passes to (group q, lane) slots: lines
// in bank order, each to the group holding the fewest lines of its bank so
// far (then the emptiest), at most 32 per group; a group then meets a bank
// conflict only where a bank holds more than LPT line starts.  The K passes
// read and write global memory and keep the natural order (slot = line), so
// that a warp's accesses for one K are 32 consecutive points; table 2 records
// that order.
template <int N>
static void line_table(std::vector<short> &tab) {
    using S = SwShape<N>;
    constexpr int NE = S::NE, LPT = S::LPT;
    tab.assign(3 * S::SLOTS, (short)-1);
    for (int id = 0; id < S::NE2; ++id) tab[2 * S::SLOTS + id] = (short)id;
    for (int ax = 0; ax < 2; ++ax) {
        std::vector<std::pair<int, int>> byb;  // (bank, line)
        for (int id = 0; id < S::NE2; ++id) {
            const int c1 = id % NE, c2 = id / NE;
            const int base = ax == 0 ? S::PJ * c1 + S::PK * c2 : ax == 1 ? c1 + S::PK * c2 : c1 + S::PJ * c2;
            byb.push_back({base % 32, id});
        }
        std::stable_sort(byb.begin(), byb.end());
        std::vector<int> size(LPT, 0), cnt(LPT * 32, 0);
        for (const auto &bl : byb) {
            int best = -1;
            for (int q = 0; q < LPT; ++q) {
                if (size[q] >= 32) continue;
                if (best < 0 || cnt[q * 32 + bl.first] < cnt[best * 32 + bl.first] ||
                    (cnt[q * 32 + bl.first] == cnt[best * 32 + bl.first] && size[q] < size[best]))
                    best = q;
            }
            tab[ax * S::SLOTS + best * 32 + size[best]] = (short)bl.second;
            ++size[best];
            ++cnt[best * 32 + bl.first];
        }
    }
}

static void line_table_n(int N, std::vector<short> &tab) {
    switch (N) {
        case 2: line_table<2>(tab); break;
        case 3: line_table<3>(tab); break;
        case 4: line_table<4>(tab); break;
        case 5: line_table<5>(tab); break;
        case 6: line_table<6>(tab); break;
        case 7: line_table<7>(tab); break;
        case 8: line_table<8>(tab); break;
        default: line_table<9>(tab); break;
    }
}

static size_t sw_layout(const sem_mesh *m, size_t *off) {
    const int ne = m->N + 3;
    const size_t P = 3 * (size_t)m->E;  // upper bound: every element and axis distinct
    const size_t nv = (size_t)coarse_topo(m).nvt;
    size_t o = 0;
    auto take = [&](size_t b) { size_t at = o; o = align_up(o + b); return at; };
    off[0] = take(sizeof(float) * P * ne * ne);
    off[1] = take(sizeof(float) * P * ne);
    off[2] = take(sizeof(int) * 3 * m->E);
    off[3] = take(sizeof(float) * (size_t)m->E * ne * ne * ne);  // also the element matrices at set-up
    off[4] = take(sizeof(float) * 8 * (size_t)m->E);
    off[5] = take(sizeof(float) * 27 * nv);
    for (int q = 6; q < 12; ++q) off[q] = take(sizeof(float) * nv);
    off[12] = take(sizeof(double) * 2 * kCgMaxGrid);
    off[13] = take(sizeof(CoarseScal));
    off[14] = take(sizeof(float) * 2 * kMaxN1);
    off[15] = take(sizeof(short) * 3 * 32 * 5);  // LPT <= 5 (N <= 9)
    return o;
}

static SwArgs sw_args(const sem_mesh *m) {
    SwArgs A;
    A.E = (int)m->E;
    for (int a = 0; a < 3; ++a) {
        A.nel[a] = m->nel[a];
        A.per[a] = m->periodic[a];
    }
    A.faces = m->faces;
    return A;
}

template <int N>
static int sw_apply_n(const sem_schwarz *sw, const float *r, float *z, int coarse_iters, double coarse_tol,
                      const int *done, cudaStream_t st, bool coop) {
    using S = SwShape<N>;
    const sem_mesh *m = sw->m;
    const SwArgs A = sw_args(m);
    const bool coarse = coarse_iters > 0;
    const size_t smem = sizeof(float) * kSwWarps * S::WARP_FLOATS + sizeof(short) * 3 * S::SLOTS;
    // resident CTAs per SM of this instantiation, queried once (concurrent
    // first callers store the same value)
    static std::atomic<int> per_sm_cache{0};
    int per_sm = per_sm_cache.load(std::memory_order_relaxed);
    if (per_sm == 0) {
        SEM_CUDA_CHECK(cudaFuncSetAttribute(schwarz_local_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
        SEM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, schwarz_local_kernel<N>,
                                                                     kSwWarps * 32, smem));
        if (per_sm < 1) per_sm = 1;
        per_sm_cache.store(per_sm, std::memory_order_relaxed);
    }
    int64_t g = (m->E + kSwWarps - 1) / kSwWarps;
    if (g > (int64_t)m->num_sms * per_sm) g = (int64_t)m->num_sms * per_sm;
    schwarz_local_kernel<N><<<(int)g, kSwWarps * 32, smem, st>>>(r, sw->S, sw->L, sw->prob, sw->J1, sw->lines, A,
                                                                  done, sw->uext, coarse ? sw->rce : nullptr);
    SEM_CUDA_CHECK(cudaGetLastError());
    const CoarseTopo C = coarse_topo(m);
    if (coarse) {
        SEM_CUDA_CHECK(cudaMemsetAsync(sw->bar, 0, sizeof(CoarseScal), st));
        CoarseArgs P;
        P.sten = sw->sten;
        P.cdinv = sw->cdinv;
        P.rce = sw->rce;
        P.x = sw->xc;
        P.r = sw->rcg;
        P.p0 = sw->pc0;
        P.p1 = sw->pc1;
        P.w = sw->wc;
        P.partial = sw->partial;
        P.bar = sw->bar;
        P.err = m->d_err;
        P.done = done;
        P.C = C;
        P.iters = coarse_iters;
        P.tol2 = coarse_tol * coarse_tol;
        static std::atomic<int> cg_cache{0};
        int cg_per_sm = cg_cache.load(std::memory_order_relaxed);
        if (cg_per_sm == 0) {
            SEM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cg_per_sm, coarse_cg_kernel, kCgThreads, 0));
            cg_cache.store(cg_per_sm, std::memory_order_relaxed);
        }
        int gc = (C.nvt + kCgThreads - 1) / kCgThreads;
        gc = std::min(gc, std::min(m->num_sms * std::max(cg_per_sm, 1), kCgMaxGrid));
        gc = std::min(gc, m->num_sms);
        if (coop) {
            void *args[] = {&P};
            SEM_CUDA_CHECK(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(coarse_cg_kernel), dim3(gc),
                                                       dim3(kCgThreads), args, 0, st));
        } else {
            CoarseScal *S = reinterpret_cast<CoarseScal *>(sw->bar);
            int gm = (C.nvt + kCgThreads - 1) / kCgThreads;
            gm = std::min(gm, kCgMaxGrid);
            coarse_mk_init_kernel<<<gm, kCgThreads, 0, st>>>(P, S);
            float *pold = sw->pc0, *pnew = sw->pc1;
            for (int it = 0; it < coarse_iters; ++it) {
                coarse_mk_pw_kernel<<<gm, kCgThreads, 0, st>>>(P, S, pold, pnew);
                coarse_mk_xr_kernel<<<gm, kCgThreads, 0, st>>>(P, S, pnew);
                std::swap(pold, pnew);
            }
            SEM_CUDA_CHECK(cudaGetLastError());
        }
    }
    int64_t gp = (m->E + sum_epb<N>() - 1) / sum_epb<N>();
    if (gp > (int64_t)m->num_sms * 16) gp = (int64_t)m->num_sms * 16;
    if ((int64_t)A.nel[0] * A.nel[1] * S::NE3 < ((int64_t)1 << 31))
        schwarz_sum_kernel<N, int><<<(int)gp, 256, 0, st>>>(sw->uext, coarse ? sw->xc : nullptr, sw->J1, A, C, done,
                                                             z);
    else
        schwarz_sum_kernel<N, int64_t><<<(int)gp, 256, 0, st>>>(sw->uext, coarse ? sw->xc : nullptr, sw->J1, A, C,
                                                                 done, z);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

int schwarz_apply_f32(const sem_schwarz *sw, const float *r, float *z, int coarse_iters, double coarse_tol,
                      const int *done, cudaStream_t st, bool coop) {
    switch (sw->N) {
#define SEM_SW_CASE(n) \
    case n: return sw_apply_n<n>(sw, r, z, coarse_iters, coarse_tol, done, st, coop);
        SEM_SW_CASE(2) SEM_SW_CASE(3) SEM_SW_CASE(4) SEM_SW_CASE(5) SEM_SW_CASE(6) SEM_SW_CASE(7)
        SEM_SW_CASE(8) SEM_SW_CASE(9)
#undef SEM_SW_CASE
        default: return fail(SEM_ERR_UNSUPPORTED, "Schwarz preconditioner built for 2 <= N <= 9");
    }
}

const sem_mesh *schwarz_mesh(const sem_schwarz *sw) { return sw ? sw->m : nullptr; }

// ---------------------------------------------------------------- intermediate level
//
// The multigrid's intermediate level: the overlapping Schwarz of the order-M
// discretisation on the same elements (a Schwarz object built on the order-M
// mesh), reached by element-wise interpolation between the GLL point sets:
//   z += w P_M S_M P_M^T r,  P_M^T r = Q_M Q_M^T J^T (r / mult_N) (masked),
// with J[i][a] = l^M_a(xi^N_i).  One CTA per element (grid-stride), the three
// 1-D contractions through shared memory, every sum in a fixed order; J's
// end rows are exact unit vectors, so the copies of a face point of the
// prolongation are bit-identical (z stays continuous).

struct MidJ {
    float J[kMaxN1 * kMaxN1];  // J[i * (M+1) + a]
};
constexpr int kMidThreads = 256;
constexpr int kMidEpb = 4;  // elements per CTA and pass: 4 consecutive slabs, coalesced

// P_M^T r element-wise (before the order-M gather-scatter): rm = J^T J^T J^T
// (r / mult), the three contractions through shared memory for kMidEpb
// elements at a time; J in shared memory.
template <int N, int M>
__global__ void __launch_bounds__(kMidThreads)
    mid_restrict_kernel(const float *__restrict__ r, const float *__restrict__ minv, const MidJ Jp, int64_t E,
                        const int *__restrict__ done, float *__restrict__ rm) {
    if (done && *done) return;
    constexpr int N1 = N + 1, M1 = M + 1, NPT = N1 * N1 * N1, MPT = M1 * M1 * M1, B = kMidEpb;
    __shared__ float sJ[N1 * M1];
    __shared__ float sa[B * NPT], s1[B * N1 * N1 * M1], s2[B * N1 * M1 * M1];
    for (int q = threadIdx.x; q < N1 * M1; q += blockDim.x) sJ[q] = Jp.J[q];
    const int64_t G = (E + B - 1) / B;
    for (int64_t g = blockIdx.x; g < G; g += gridDim.x) {
        const int64_t e0 = g * B;
        const int nv = (int)((E - e0) < B ? (E - e0) : B);
        __syncthreads();
        for (int q = threadIdx.x; q < nv * NPT; q += blockDim.x) sa[q] = r[e0 * NPT + q] * minv[e0 * NPT + q];
        __syncthreads();
        for (int q = threadIdx.x; q < nv * N1 * N1 * M1; q += blockDim.x) {  // (e, k, j, a): over i
            const int a = q % M1, ekj = q / M1;
            float t = 0.f;
#pragma unroll
            for (int i = 0; i < N1; ++i) t = fmaf(sJ[i * M1 + a], sa[ekj * N1 + i], t);
            s1[q] = t;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < nv * N1 * M1 * M1; q += blockDim.x) {  // (e, k, b, a): over j
            const int a = q % M1, b = (q / M1) % M1, ek = q / (M1 * M1);
            float t = 0.f;
#pragma unroll
            for (int j = 0; j < N1; ++j) t = fmaf(sJ[j * M1 + b], s1[(ek * N1 + j) * M1 + a], t);
            s2[q] = t;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < nv * MPT; q += blockDim.x) {  // (e, c, b, a): over k
            const int ba = q % (M1 * M1), c = (q / (M1 * M1)) % M1, el = q / MPT;
            float t = 0.f;
#pragma unroll
            for (int k = 0; k < N1; ++k) t = fmaf(sJ[k * M1 + c], s2[(el * N1 + k) * M1 * M1 + ba], t);
            rm[e0 * MPT + q] = t;
        }
    }
}

// z += w P_M zm element-wise (zm continuous: the copies of a face point get
// the same bits, J's end rows being exact unit vectors).
template <int N, int M>
__global__ void __launch_bounds__(kMidThreads)
    mid_prolong_add_kernel(const float *__restrict__ zm, const MidJ Jp, float w, int64_t E,
                           const int *__restrict__ done, float *__restrict__ z) {
    if (done && *done) return;
    constexpr int N1 = N + 1, M1 = M + 1, NPT = N1 * N1 * N1, MPT = M1 * M1 * M1, B = kMidEpb;
    __shared__ float sJ[N1 * M1];
    __shared__ float s0[B * MPT], s1[B * M1 * M1 * N1], s2[B * M1 * N1 * N1];
    for (int q = threadIdx.x; q < N1 * M1; q += blockDim.x) sJ[q] = Jp.J[q];
    const int64_t G = (E + B - 1) / B;
    for (int64_t g = blockIdx.x; g < G; g += gridDim.x) {
        const int64_t e0 = g * B;
        const int nv = (int)((E - e0) < B ? (E - e0) : B);
        __syncthreads();
        for (int q = threadIdx.x; q < nv * MPT; q += blockDim.x) s0[q] = zm[e0 * MPT + q];
        __syncthreads();
        for (int q = threadIdx.x; q < nv * M1 * M1 * N1; q += blockDim.x) {  // (e, c, b, i): over a
            const int i = q % N1, ecb = q / N1;
            float t = 0.f;
#pragma unroll
            for (int a = 0; a < M1; ++a) t = fmaf(sJ[i * M1 + a], s0[ecb * M1 + a], t);
            s1[q] = t;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < nv * M1 * N1 * N1; q += blockDim.x) {  // (e, c, j, i): over b
            const int i = q % N1, j = (q / N1) % N1, ec = q / (N1 * N1);
            float t = 0.f;
#pragma unroll
            for (int b = 0; b < M1; ++b) t = fmaf(sJ[j * M1 + b], s1[(ec * M1 + b) * N1 + i], t);
            s2[q] = t;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < nv * NPT; q += blockDim.x) {  // (e, k, j, i): over c
            const int ji = q % (N1 * N1), k = (q / (N1 * N1)) % N1, el = q / NPT;
            float t = 0.f;
#pragma unroll
            for (int c = 0; c < M1; ++c) t = fmaf(sJ[k * M1 + c], s2[(el * M1 + c) * N1 * N1 + ji], t);
            z[e0 * NPT + q] = fmaf(w, t, z[e0 * NPT + q]);
        }
    }
}

template <int N, int M>
static int mid_launch_nm(bool prolong, const float *in, const float *minv, const MidJ &J, float w, int64_t E,
                         int num_sms, const int *done, float *out, cudaStream_t st) {
    const int64_t G = (E + kMidEpb - 1) / kMidEpb;
    const int grid = (int)(G < (int64_t)num_sms * 8 ? G : (int64_t)num_sms * 8);
    if (prolong)
        mid_prolong_add_kernel<N, M><<<grid, kMidThreads, 0, st>>>(in, J, w, E, done, out);
    else
        mid_restrict_kernel<N, M><<<grid, kMidThreads, 0, st>>>(in, minv, J, E, done, out);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

template <int N>
static int mid_launch_n(int M, bool prolong, const float *in, const float *minv, const MidJ &J, float w, int64_t E,
                        int num_sms, const int *done, float *out, cudaStream_t st) {
    switch (M) {
#define SEM_MID_M(mm) \
    case mm:           \
        if constexpr (mm < N) return mid_launch_nm<N, mm>(prolong, in, minv, J, w, E, num_sms, done, out, st); \
        break;
        SEM_MID_M(2) SEM_MID_M(3) SEM_MID_M(4) SEM_MID_M(5) SEM_MID_M(6) SEM_MID_M(7) SEM_MID_M(8)
#undef SEM_MID_M
        default: break;
    }
    return fail(SEM_ERR_UNSUPPORTED, "intermediate order outside 2 <= M < N");
}

static int mid_launch(int N, int M, bool prolong, const float *in, const float *minv, const MidJ &J, float w,
                      int64_t E, int num_sms, const int *done, float *out, cudaStream_t st) {
    switch (N) {
#define SEM_MID_N(nn) \
    case nn: return mid_launch_n<nn>(M, prolong, in, minv, J, w, E, num_sms, done, out, st);
        SEM_MID_N(3) SEM_MID_N(4) SEM_MID_N(5) SEM_MID_N(6) SEM_MID_N(7) SEM_MID_N(8) SEM_MID_N(9)
#undef SEM_MID_N
        default: return fail(SEM_ERR_UNSUPPORTED, "intermediate level built for 3 <= N <= 9");
    }
}

// J[i][a] = l^M_a(xi^N_i) by Lagrange's product formula (host, FP64).
static void mid_interp(const sem_mesh *fine, const sem_mesh *mid, MidJ &out) {
    const int N1 = fine->N + 1, M1 = mid->N + 1;
    for (int q = 0; q < kMaxN1 * kMaxN1; ++q) out.J[q] = 0.f;
    for (int i = 0; i < N1; ++i) {
        const double x = fine->xi[i];
        int hit = -1;
        for (int a = 0; a < M1; ++a)
            if (std::fabs(x - mid->xi[a]) < 1e-14) hit = a;
        for (int a = 0; a < M1; ++a) {
            double v = 1.0;
            if (hit >= 0) {
                v = a == hit ? 1.0 : 0.0;
            } else {
                for (int b = 0; b < M1; ++b)
                    if (b != a) v *= (x - mid->xi[b]) / (mid->xi[a] - mid->xi[b]);
            }
            out.J[i * M1 + a] = (float)v;
        }
    }
}

size_t schwarz_mid_work_bytes(const sem_schwarz *mid) {
    return mid ? 2 * align_up(sizeof(float) * mid->m->nloc) : 0;
}

// The same elements and topology, a lower order, both Schwarz objects on
// meshes of their own (else SEM_ERR_INVALID_ARG).
int schwarz_mid_check(const sem_schwarz *sw, const sem_schwarz *mid) {
    if (!sw || !mid) return fail(SEM_ERR_INVALID_ARG, "NULL Schwarz object");
    const sem_mesh *f = sw->m, *m = mid->m;
    if (m->N >= f->N || m->E != f->E || m->faces != f->faces)
        return fail(SEM_ERR_INVALID_ARG, "the intermediate level needs a lower order on the same elements");
    for (int a = 0; a < 3; ++a)
        if (m->nel[a] != f->nel[a] || m->periodic[a] != f->periodic[a])
            return fail(SEM_ERR_INVALID_ARG, "the intermediate level needs the same topology");
    return SEM_OK;
}

// z += w P_M S_M P_M^T r (FP32; work: schwarz_mid_work_bytes; done: guard).
int schwarz_mid_apply_add(const sem_schwarz *sw, const sem_schwarz *mid, double w, const float *r, float *z,
                          void *work, const int *done, cudaStream_t st) {
    const sem_mesh *f = sw->m, *m = mid->m;
    MidJ J;
    mid_interp(f, m, J);
    float *rm = static_cast<float *>(work);
    float *zm = reinterpret_cast<float *>(static_cast<char *>(work) + align_up(sizeof(float) * m->nloc));
    int s = mid_launch(f->N, m->N, false, r, f->minv32, J, 0.f, f->E, f->num_sms, done, rm, st);
    if (s != SEM_OK) return s;
    s = gs_launch(m, rm, SEM_F32, kGsSumMask, st, done, 0);
    if (s != SEM_OK) return s;
    s = schwarz_apply_f32(mid, rm, zm, 0, 0.0, done, st);
    if (s != SEM_OK) return s;
    return mid_launch(f->N, m->N, true, zm, nullptr, J, (float)w, f->E, f->num_sms, done, z, st);
}

}  // namespace sem

using namespace sem;

extern "C" {

size_t sem_schwarz_workspace_bytes(const sem_mesh *m, const sem_mesh *mc) {
    if (!m || !mc) return 0;
    size_t off[16];
    return sw_layout(m, off);
}

int sem_schwarz_create(const sem_mesh *m, const sem_mesh *mc, void *ws, size_t bytes, void *stream,
                       sem_schwarz **out) {
    if (!m || !mc || !out) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (m->N < 2 || m->N > 9) return fail(SEM_ERR_UNSUPPORTED, "Schwarz preconditioner built for 2 <= N <= 9");
    if (!m->G32) return fail(SEM_ERR_INVALID_ARG, "the mesh needs SEM_GEOM_F32");
    if (mc->N != 1 || mc->E != m->E)
        return fail(SEM_ERR_INVALID_ARG, "the coarse mesh must be the N = 1 mesh of the same elements");
    for (int a = 0; a < 3; ++a)
        if (mc->nel[a] != m->nel[a] || mc->periodic[a] != m->periodic[a])
            return fail(SEM_ERR_INVALID_ARG, "the coarse mesh must have the same topology");
    size_t off[16];
    const size_t need = sw_layout(m, off);
    if (!ws || reinterpret_cast<uintptr_t>(ws) % kAlign || bytes < need)
        return fail(SEM_ERR_WORKSPACE, "Schwarz workspace NULL, misaligned or smaller than sem_schwarz_workspace_bytes");
    cudaStream_t st = as_stream(stream);
    const int N = m->N, n1 = N + 1, ne = N + 3;
    const int64_t E = m->E;
    // element lengths from the vertices (mean edge length per direction)
    std::vector<double> V(24 * E);
    SEM_CUDA_CHECK(cudaMemcpyAsync(V.data(), m->verts, sizeof(double) * 24 * E, cudaMemcpyDeviceToHost, st));
    SEM_CUDA_CHECK(cudaStreamSynchronize(st));
    std::vector<double> hl[3];
    for (int a = 0; a < 3; ++a) hl[a].resize(E);
    static const int edges[3][4] = {{0, 2, 4, 6}, {0, 1, 4, 5}, {0, 1, 2, 3}};
    static const int step[3] = {1, 2, 4};
    for (int64_t e = 0; e < E; ++e)
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int q = 0; q < 4; ++q) {
                const double *p0 = &V[24 * e + 3 * edges[a][q]], *p1 = &V[24 * e + 3 * (edges[a][q] + step[a])];
                s += std::sqrt((p1[0] - p0[0]) * (p1[0] - p0[0]) + (p1[1] - p0[1]) * (p1[1] - p0[1]) +
                               (p1[2] - p0[2]) * (p1[2] - p0[2]));
            }
            hl[a][e] = 0.25 * s;
        }
    // reference 1-D stiffness and mass
    std::vector<double> Ah(n1 * n1, 0.0), Bh(n1, 0.0);
    ref_1d(N, m->rho, m->D.d, Ah.data(), Bh.data());
    std::map<FdmKey, int> cache;
    std::vector<float> Stab, Ltab;
    std::vector<int> prob(3 * E);
    const int stride[3] = {1, m->nel[0], m->nel[0] * m->nel[1]};
    std::vector<double> Sd(ne * ne), ld(ne);
    for (int64_t e = 0; e < E; ++e) {
        const int coord[3] = {(int)(e % m->nel[0]), (int)((e / m->nel[0]) % m->nel[1]),
                              (int)(e / ((int64_t)m->nel[0] * m->nel[1]))};
        for (int a = 0; a < 3; ++a) {
            const int c = coord[a], n = m->nel[a], per = m->periodic[a];
            const bool hasL = c > 0 || per, hasR = c < n - 1 || per;
            const bool dirL = !per && c == 0 && ((m->faces >> (2 * a)) & 1);
            const bool dirR = !per && c == n - 1 && ((m->faces >> (2 * a + 1)) & 1);
            const int64_t eL = c > 0 ? e - stride[a] : e + (int64_t)(n - 1) * stride[a];
            const int64_t eR = c < n - 1 ? e + stride[a] : e - (int64_t)(n - 1) * stride[a];
            const double h = hl[a][e], hL = hasL ? hl[a][eL] : h, hR = hasR ? hl[a][eR] : h;
            const FdmKey key{qlen(h), qlen(hL), qlen(hR),
                             (hasL ? 1 : 0) | (hasR ? 2 : 0) | (dirL ? 4 : 0) | (dirR ? 8 : 0)};
            auto it = cache.find(key);
            if (it != cache.end()) {
                prob[3 * e + a] = it->second;
                continue;
            }
            fdm_1d(N, Ah.data(), Bh.data(), h, hL, hR, hasL, hasR, dirL, dirR, Sd.data(), ld.data());
            const int id = (int)(Ltab.size() / ne);
            for (int q = 0; q < ne * ne; ++q) Stab.push_back((float)Sd[q]);
            for (int q = 0; q < ne; ++q) Ltab.push_back((float)ld[q]);
            cache[key] = id;
            prob[3 * e + a] = id;
        }
    }
    sem_schwarz *sw = new (std::nothrow) sem_schwarz();
    if (!sw) return fail(SEM_ERR_INVALID_ARG, "host allocation failed");
    char *base = static_cast<char *>(ws);
    sw->m = m;
    sw->mc = mc;
    sw->N = N;
    sw->ne = ne;
    sw->P = (int)(Ltab.size() / ne);
    sw->S = reinterpret_cast<float *>(base + off[0]);
    sw->L = reinterpret_cast<float *>(base + off[1]);
    sw->prob = reinterpret_cast<int *>(base + off[2]);
    sw->uext = reinterpret_cast<float *>(base + off[3]);
    sw->rce = reinterpret_cast<float *>(base + off[4]);
    sw->sten = reinterpret_cast<float *>(base + off[5]);
    float *cv[6];
    for (int q = 0; q < 6; ++q) cv[q] = reinterpret_cast<float *>(base + off[6 + q]);
    sw->cdinv = cv[0];
    sw->xc = cv[1];
    sw->rcg = cv[2];
    sw->pc0 = cv[3];
    sw->pc1 = cv[4];
    sw->wc = cv[5];
    sw->partial = reinterpret_cast<double *>(base + off[12]);
    sw->bar = reinterpret_cast<unsigned *>(base + off[13]);
    sw->J1 = reinterpret_cast<float *>(base + off[14]);
    sw->lines = reinterpret_cast<short *>(base + off[15]);
    std::vector<short> ltab;
    line_table_n(N, ltab);
    const CoarseTopo C = coarse_topo(m);
    sw->nv = C.nvt;
    sw->ws_bytes = need;
    std::vector<float> J1(2 * kMaxN1, 0.f);
    for (int i = 0; i <= N; ++i) {
        J1[i] = (float)(0.5 * (1.0 - m->xi[i]));
        J1[kMaxN1 + i] = (float)(0.5 * (1.0 + m->xi[i]));
    }
    cudaError_t ce = cudaMemcpyAsync(sw->S, Stab.data(), sizeof(float) * Stab.size(), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(sw->L, Ltab.data(), sizeof(float) * Ltab.size(), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(sw->prob, prob.data(), sizeof(int) * prob.size(), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(sw->J1, J1.data(), sizeof(float) * J1.size(), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(sw->lines, ltab.data(), sizeof(short) * ltab.size(), cudaMemcpyHostToDevice, st);
    // the coarse operator: N = 1 element matrices (in the extended-solution
    // buffer, free until the first application), then the vertex stencil
    if (ce == cudaSuccess) {
        const int64_t tE = 8 * E;
        coarse_elem_kernel<<<(int)std::min<int64_t>((tE + 255) / 256, 4096), 256, 0, st>>>(mc->G, (int)E, sw->uext);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) {
        coarse_stencil_kernel<<<std::min((C.nvt + 255) / 256, 4096), 256, 0, st>>>(sw->uext, C, sw->sten, sw->cdinv);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
        delete sw;
        return cuda_fail(ce, "sem_schwarz_create upload");
    }
    *out = sw;
    return SEM_OK;
}

int sem_schwarz_destroy(sem_schwarz *sw) {
    delete sw;
    return SEM_OK;
}

int sem_schwarz_problems(const sem_schwarz *sw) { return sw ? sw->P : -1; }

int sem_schwarz_fdm_1d(int N, double h, double hL, double hR, int flags, double *S, double *lambda) {
    if (N < 2 || N > 9) return fail(SEM_ERR_UNSUPPORTED, "Schwarz preconditioner built for 2 <= N <= 9");
    if (!S || !lambda || !(h > 0.0) || !(hL > 0.0) || !(hR > 0.0) || (flags & ~15))
        return fail(SEM_ERR_INVALID_ARG, "NULL output, non-positive length or unknown flag");
    double xi[kMaxN1], rho[kMaxN1], D[kMaxN1 * kMaxN1], Ah[kMaxN1 * kMaxN1], Bh[kMaxN1];
    gll_host(N, xi, rho);
    deriv_host(N, xi, D);
    ref_1d(N, rho, D, Ah, Bh);
    fdm_1d(N, Ah, Bh, h, hL, hR, flags & 1, flags & 2, flags & 4, flags & 8, S, lambda);
    return SEM_OK;
}

int sem_schwarz_coarse_operator(const int *nel, const int *periodic, int faces, const double *G, float *sten,
                                float *cdinv) {
    if (!nel || !periodic || !G || !sten || !cdinv) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    for (int a = 0; a < 3; ++a)
        if (nel[a] < 1) return fail(SEM_ERR_INVALID_ARG, "nel < 1");
    const CoarseTopo C = coarse_topo(nel, periodic, faces);
    const int64_t E = (int64_t)nel[0] * nel[1] * nel[2];
    std::vector<float> Ae(64 * E);
    for (int64_t e = 0; e < E; ++e)
        for (int j = 0; j < 8; ++j) coarse_elem_col(G + e * 48, j, Ae.data() + e * 64);
    for (int v = 0; v < C.nvt; ++v) coarse_stencil_row(Ae.data(), C, v, sten, cdinv);
    return SEM_OK;
}

int sem_schwarz_line_table(int N, short *out, int cap, int *slots, int *pj, int *pk) {
    if (N < 2 || N > 9) return fail(SEM_ERR_UNSUPPORTED, "Schwarz preconditioner built for 2 <= N <= 9");
    if (!out || !slots || !pj || !pk) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    std::vector<short> t;
    line_table_n(N, t);
    if (cap < (int)t.size()) return fail(SEM_ERR_WORKSPACE, "line table larger than cap");
    std::copy(t.begin(), t.end(), out);
    *slots = (int)t.size() / 3;
    switch (N) {
#define SEM_LT_CASE(n)              \
    case n:                         \
        *pj = SwShape<n>::PJ;       \
        *pk = SwShape<n>::PK;       \
        break;
        SEM_LT_CASE(2) SEM_LT_CASE(3) SEM_LT_CASE(4) SEM_LT_CASE(5) SEM_LT_CASE(6) SEM_LT_CASE(7)
        SEM_LT_CASE(8) SEM_LT_CASE(9)
#undef SEM_LT_CASE
    }
    return SEM_OK;
}

int sem_schwarz_apply(const sem_schwarz *sw, const float *r, float *z, int coarse_iters, double coarse_tol,
                      void *stream) {
    NvtxRange nvtx_range("Schwarz application");
    if (!sw || !r || !z) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    if (r == z) return fail(SEM_ERR_INVALID_ARG, "r and z must not overlap");
    if (coarse_iters < 0) return fail(SEM_ERR_INVALID_ARG, "coarse_iters < 0");
    return schwarz_apply_f32(sw, r, z, coarse_iters, coarse_tol, nullptr, as_stream(stream));
}

size_t sem_schwarz_mid_work_bytes(const sem_schwarz *mid) { return schwarz_mid_work_bytes(mid); }

int sem_schwarz_apply3(const sem_schwarz *sw, const sem_schwarz *mid, double mid_weight, const float *r, float *z,
                       int coarse_iters, double coarse_tol, void *d_work, size_t bytes, void *stream) {
    if (!sw || !r || !z) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    if (r == z) return fail(SEM_ERR_INVALID_ARG, "r and z must not overlap");
    if (coarse_iters < 0) return fail(SEM_ERR_INVALID_ARG, "coarse_iters < 0");
    int s = schwarz_mid_check(sw, mid);
    if (s != SEM_OK) return s;
    if (!(mid_weight > 0.0)) return fail(SEM_ERR_INVALID_ARG, "mid_weight must be > 0");
    if (!d_work || bytes < schwarz_mid_work_bytes(mid) || reinterpret_cast<uintptr_t>(d_work) % kAlign)
        return fail(SEM_ERR_WORKSPACE, "work smaller than sem_schwarz_mid_work_bytes or misaligned");
    cudaStream_t st = as_stream(stream);
    s = schwarz_apply_f32(sw, r, z, coarse_iters, coarse_tol, nullptr, st);
    if (s != SEM_OK) return s;
    return schwarz_mid_apply_add(sw, mid, mid_weight, r, z, d_work, nullptr, st);
}

}  // extern "C"
