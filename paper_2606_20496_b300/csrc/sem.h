// Spectral-element levels of the p-multigrid wrap (Sec. 1, Sec. 5, Eqs. (13)
// and (14)): host set-up (sem_setup.cpp), kernels and launchers (sem.cu).
//
// A level of order n has p = n + 1 Gauss-Lobatto-Legendre (GLL) nodes per
// direction.  Element-local data are [element][k][j][i] with i fastest
// (lexicographic, Sec. 1); hexahedron vertex a + 2b + 4c is the local node
// (a n, b n, c n).  Global node numbers start with the mesh vertices (so the
// order-1 level is the vertex numbering itself), then the nodes inside edges,
// inside faces and inside elements.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

namespace cgs {

constexpr int kSemMinOrder = 2;
constexpr int kSemMaxOrder = 8;

// 1D GLL rule and operators of order n (sem_setup.cpp).
void gll_rule(int n, std::vector<double>& x, std::vector<double>& w);
// D[i * p + j] = l_j'(x_i)
void gll_derivative(int n, const std::vector<double>& x, std::vector<double>& D);
// I[i * pc + j] = l_j(xf_i) for the Lagrange basis on xc
void lagrange_interp(const std::vector<double>& xc, const std::vector<double>& xf, std::vector<double>& I);

// One level on the host, before upload.
struct SemHostLevel {
    int n = 0, p = 0;
    int64_t ng = 0;                 // global nodes
    int64_t nfree = 0;              // of them not Dirichlet
    std::vector<int32_t> l2g;       // ne * p^3 global node of every element-local node
    std::vector<double> G;          // ne * 6 * p^3: w det J (J^-1 J^-T), entries 00 01 02 11 12 22
    std::vector<uint8_t> dir;       // ng
    std::vector<double> inv_mult;   // ng: 1 / elements holding the node
    std::vector<double> S;          // ne * 3 * p * p: per direction S_d[node * p + mode]
    std::vector<double> lam;        // ne * 3 * p
    std::vector<double> D;          // p * p
    std::vector<double> x;          // p GLL nodes
};

// Build a level of order n (2..8) from the hexahedral mesh; `vdir` is the
// vertex Dirichlet mask (boundary-face vertices).  Returns an empty string
// or the reason for failure.
std::string sem_build_level(int n, const double* xyz, int64_t nv, const int32_t* conn, int64_t ne,
                            SemHostLevel& L);
// Vertex Dirichlet mask of the default set: every vertex of a face owned by
// one element.
std::vector<uint8_t> sem_boundary_vertices(const int32_t* conn, int64_t ne, int64_t nv);
// Coordinates of a level's global nodes (trilinear map of each element).
void sem_node_coords(int n, const double* xyz, const int32_t* conn, int64_t ne, const std::vector<int32_t>& l2g,
                     int64_t ng, double* out);

// One level on the device.
struct SemDevLevel {
    int n = 0, p = 0;
    int64_t ng = 0, nfree = 0;
    int32_t* l2g = nullptr;         // a Dirichlet node g is stored as -(g + 1)
    double* G = nullptr;
    uint8_t* dir = nullptr;
    double* inv_mult = nullptr;
    double* S = nullptr;
    double* lam = nullptr;
    double* D = nullptr;
    double* I_next = nullptr;       // p x p_next interpolation to the next (coarser) level
    // float copies for the float smoother and transfers (f32 set)
    bool f32 = false;
    float* S32 = nullptr;
    float* lam32 = nullptr;
    float* inv_mult32 = nullptr;
    float* I_next32 = nullptr;
    float2* Gp = nullptr;           // metric as (hi, lo) pairs: the pair operator (f32 set)
    float2* Dp = nullptr;           // D as pairs
    void* r = nullptr;              // work vectors of this level (levels below the finest):
    void* z = nullptr;              // float when f32, else float64
};

// Launchers (sem.cu).  Dirichlet entries are skipped on input and never
// written.  Vector types: float64, or float where the flag says so (only
// with L.f32 / F.f32).
// y += A_n x (float64; y cleared by the caller)
void launch_sem_ax(const SemDevLevel& L, int64_t ne, const double* x, double* y, cudaStream_t st);
// z += W sum_e R_e^T A~_e^-1 R_e r (Eq. (14))
void launch_sem_fdm(const SemDevLevel& L, int64_t ne, const void* r, void* z, bool vec_f32, cudaStream_t st);
// rc += J^T rf = Q_c^T I^T Q_f W_f rf; coarse l2g of pc^3 entries per element
void launch_sem_restrict(const SemDevLevel& F, int pc, const int32_t* l2g_c, int64_t ne, const void* rf, void* rc,
                         bool f_f32, bool c_f32, cudaStream_t st);
// zf += J uc = W_f Q_f^T I Q_c uc
void launch_sem_prolong(const SemDevLevel& F, int pc, const int32_t* l2g_c, int64_t ne, const void* uc, void* zf,
                        bool c_f32, bool f_f32, cudaStream_t st);

}  // namespace cgs
