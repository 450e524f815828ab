// hx_core.cuh -- per-degree body of the operator kernels, included once per
// (degree, precision) by hx_ops.cu and once per degree by hx_batch.cu. The
// includer defines HX_P, HX_UNIT_F32 and the scalar type Real and opens the
// enclosing namespaces; this file has no include guard on purpose.
//
// Per element the operators follow the same pipeline (Sec. 2 weak forms,
// sum factorization as in the paper's matrix-free setting, Sec. 6):
//   gather      x-rows of u_e <- u[conn(e)] into registers
//   interpolate V = (B (x) B (x) B) u_e                  three 1D sweeps
//   gradient    dV/dxi_d = D_d V (collocation on the Gauss points, q = p+1)
//   qp operator H = (dV/dxi) J0^-1, material law, Q = JxW * dP J0^-T
//   integrate   r_e = sum_d D_d^T Q_d, then (B^T (x) B^T (x) B^T)
//   scatter     out[conn(e)] += r_e  (atomic adds into a zeroed vector)

constexpr int N = HX_P + 1;        // nodes (and Gauss points) per direction
constexpr int NN = N * N;
constexpr int NQ = N * N * N;      // nodes (and Gauss points) per element
constexpr int R = (N % 2) ? N : N + 1;  // padded row length (odd)
constexpr int SZ = R * N * N;      // padded cube size

// Column-layout cubes of the apply kernel: element e of an array starts at
// e*ES, component c at +c*CZ, point (i,j,k) at +i + j*RS + k*PS. The strides
// were chosen by an exhaustive bank-conflict search over the three line-sweep
// access patterns of a warp (lanes spanning several elements), separately for
// 4- and 8-byte words.
struct ColLayout {
    int RS, PS, CZ, ES;
};
constexpr ColLayout col_layout() {
    if (sizeof(Real) == 4) {
        return N == 2 ? ColLayout{2, 5, 10, 36}
             : N == 3 ? ColLayout{3, 14, 42, 137}
             : N == 4 ? ColLayout{4, 19, 76, 240}
             : N == 5 ? ColLayout{5, 25, 125, 377}
             : N == 6 ? ColLayout{7, 42, 252, 764}
                      : ColLayout{7, 56, 392, 1201};
    }
    return N == 2 ? ColLayout{2, 5, 10, 36}
         : N == 3 ? ColLayout{3, 18, 54, 169}
         : N == 4 ? ColLayout{4, 19, 76, 228}
         : N == 5 ? ColLayout{5, 25, 125, 377}
         : N == 6 ? ColLayout{9, 54, 324, 980}
                  : ColLayout{7, 52, 364, 1105};
}
constexpr int CRS = col_layout().RS, CPS = col_layout().PS, CCZ = col_layout().CZ, CES = col_layout().ES;

enum { TB = 0, TD = 1, TG = 2 };

// threads per CTA of the column-layout apply: n^2 threads per element
__host__ __device__ constexpr int col_threads(int epb) { return (epb * NN + 31) / 32 * 32; }

// Row-swizzled cubes of the staged FP32 apply at n = 5: every element owns a
// whole warp (25 of 32 lanes active) and the x-row (j, k) of a cube starts at
// word RS5[j][k] of its component block. The starts are distinct modulo 32
// and, along any j or any k, at least five banks apart, so the x-, y- and
// z-line sweeps (25 lanes, one word each) are free of bank conflicts; rows
// are packed into 154 words per component.
constexpr bool ROWSW = N == 5 && sizeof(Real) == 4;
__constant__ int cRS5[5][5] = {{122, 72, 127, 149, 45},
                               {39, 56, 12, 34, 50},
                               {116, 67, 89, 111, 94},
                               {1, 17, 6, 28, 23},
                               {78, 61, 83, 105, 100}};
template <bool SW>
struct Lay {
    static constexpr int CZ = SW ? 154 : CCZ;        // component stride (words)
    static constexpr int ES = SW ? 3 * 154 : CES;    // element stride (words)
};
// threads per CTA of the apply for a tile of epb elements
template <bool SW>
__host__ __device__ constexpr int apply_threads(int epb) {
    return SW ? epb * 32 : col_threads(epb);
}
// element, line coordinates and activity of thread t
template <bool SW>
__device__ __forceinline__ void thread_map(int t, int epb, int &el, int &a0, int &a1, bool &act) {
    int a;
    if constexpr (SW) {
        el = t >> 5;
        a = t & 31;
        act = a < NN && el < epb;
    } else {
        el = t / NN;
        a = t - el * NN;
        act = el < epb;
    }
    a0 = a % N;
    a1 = a / N;
}
// element-local word offsets of a thread's lines (component 0): x-line start,
// y-line points j and z-line points k
template <bool SW>
struct LineOffs {
    int x, y[N], z[N];
};
template <bool SW>
__device__ __forceinline__ LineOffs<SW> line_offsets(int a0, int a1) {
    LineOffs<SW> o;
    if constexpr (SW) {
        const int b0 = a0 < N ? a0 : 0, b1 = a1 < N ? a1 : 0;
        o.x = cRS5[b0][b1];
#pragma unroll
        for (int t = 0; t < N; ++t) {
            o.y[t] = cRS5[t][b1] + b0;
            o.z[t] = cRS5[b1][t] + b0;
        }
    } else {
        o.x = a0 * CRS + a1 * CPS;
#pragma unroll
        for (int t = 0; t < N; ++t) {
            o.y[t] = a0 + t * CRS + a1 * CPS;
            o.z[t] = a0 + a1 * CRS + t * CPS;
        }
    }
    return o;
}

// threads per CTA for a tile of epb elements: one thread per sweep line
__host__ __device__ constexpr int threads_for(int epb) {
    return (3 * epb * NN + 31) / 32 * 32 < 64 ? 64 : ((3 * epb * NN + 31) / 32 * 32 > 1024 ? 1024 : (3 * epb * NN + 31) / 32 * 32);
}

__constant__ Real cTab[3][NN];       // B[q][a], D[q][r], Gd[q][a]
// Even-odd halves of the 1D matrices. On points symmetric about 1/2, B is
// symmetric and D, Gd antisymmetric under (o, t) -> (N-1-o, N-1-t); for
// o, t < N/2, P = (M[o][t] + M[o][N-1-t]) / 2 and Q = (M[o][t] - M[o][N-1-t]) / 2
// of M and of M^T: [table][transposed][P, Q][o * (N/2) + t]
constexpr int EOH = N / 2;
__constant__ Real cEO[3][2][2][(EOH > 0 ? EOH : 1) * (EOH > 0 ? EOH : 1)];
__constant__ double cW[N];           // Gauss weights on [0,1]
__constant__ double cGeoV[2][3 * N]; // geometry bases at Gauss points [g-1][a*N+q]
__constant__ double cGeoD[2][3 * N];
__constant__ double cGeoVn[2][3 * N];  // geometry bases at the nodal points

template <int TAB>
__device__ __forceinline__ Real tab(int i) {
    return cTab[TAB][i];
}

__device__ __forceinline__ int cidx(int i, int j, int k) { return i + R * (j + N * k); }

// sym6 index of (i,j): xx yy zz xy xz yz
__host__ __device__ constexpr int SI(int i, int j) {
    return (i == j) ? i : ((i + j == 1) ? 3 : ((i + j == 2) ? 4 : 5));
}

// ---------------------------------------------------------------------------
// 1D line sweeps over padded cubes in shared memory. Lines along DIR of cube
// (cube*IM + IO) are contracted with table TAB (transposed if TR) and written
// (or added, ACC) to cube (cube*OM + OO). One thread per line, register
// blocked: N loads, N*N FMAs, N stores.
// ---------------------------------------------------------------------------
template <typename T, int DIR, int TAB, bool TR, bool ACC, int IM, int IO, int OM, int OO>
__device__ __forceinline__ void sweep(const T *__restrict__ in, T *__restrict__ out, int ncubes) {
    const int nlines = ncubes * NN;
    for (int l = threadIdx.x; l < nlines; l += blockDim.x) {
        const int cube = l / NN;
        const int r = l - cube * NN;
        const int a = r % N, b = r / N;
        int off, str;
        if constexpr (DIR == 0) {
            off = R * (a + N * b);
            str = 1;
        } else if constexpr (DIR == 1) {
            off = a + R * N * b;
            str = R;
        } else {
            off = a + R * b;
            str = R * N;
        }
        const T *ip = in + (cube * IM + IO) * SZ + off;
        T *op = out + (cube * OM + OO) * SZ + off;
        T x[N];
#pragma unroll
        for (int t = 0; t < N; ++t) x[t] = ip[t * str];
#pragma unroll
        for (int o = 0; o < N; ++o) {
            T s = T(0);
#pragma unroll
            for (int t = 0; t < N; ++t) s = fma((T)tab<TAB>(TR ? t * N + o : o * N + t), x[t], s);
            if constexpr (ACC)
                op[o * str] += s;
            else
                op[o * str] = s;
        }
    }
}

// values u_e (3*EPB cubes in U) -> reference gradients at Gauss points in G
// (cube (e*3+c)*3+d holds d u_c / d xi_d). W is scratch; U is clobbered.
template <typename T>
__device__ __forceinline__ void forward_grad(T *U, T *W, T *G, int nc) {
    sweep<T, 0, TB, false, false, 1, 0, 1, 0>(U, W, nc);
    __syncthreads();
    sweep<T, 1, TB, false, false, 1, 0, 1, 0>(W, U, nc);
    __syncthreads();
    sweep<T, 2, TB, false, false, 1, 0, 1, 0>(U, W, nc);
    __syncthreads();
    sweep<T, 0, TD, false, false, 1, 0, 3, 0>(W, G, nc);
    sweep<T, 1, TD, false, false, 1, 0, 3, 1>(W, G, nc);
    sweep<T, 2, TD, false, false, 1, 0, 3, 2>(W, G, nc);
    __syncthreads();
}

// test-gradient integration: G (per-qp coefficients Q_{c,d}) -> nodal values in U
template <typename T>
__device__ __forceinline__ void backward_int(T *G, T *W, T *U, int nc) {
    sweep<T, 0, TD, true, false, 3, 0, 1, 0>(G, W, nc);
    __syncthreads();
    sweep<T, 1, TD, true, true, 3, 1, 1, 0>(G, W, nc);
    __syncthreads();
    sweep<T, 2, TD, true, true, 3, 2, 1, 0>(G, W, nc);
    __syncthreads();
    sweep<T, 2, TB, true, false, 1, 0, 1, 0>(W, U, nc);
    __syncthreads();
    sweep<T, 1, TB, true, false, 1, 0, 1, 0>(U, W, nc);
    __syncthreads();
    sweep<T, 0, TB, true, false, 1, 0, 1, 0>(W, U, nc);
    __syncthreads();
}

// ---------------------------------------------------------------------------
// gather / scatter
// ---------------------------------------------------------------------------
// n / d for 0 <= n < 2^31 (see hx::FastDiv)
__device__ __forceinline__ int fast_div(int n, const hx::FastDiv &f) {
    const uint32_t t = __umulhi(f.m, (uint32_t)n);
    return (int)((t + (((uint32_t)n - t) >> f.s1)) >> f.s2);
}
// element lattice indices of element e of a structured box
__device__ __forceinline__ void elem_xyz(const hx::MeshView &m, int e, int &ex, int &ey, int &ez) {
    const int t = fast_div(e, m.fnx);
    ex = e - t * m.nx;
    ez = fast_div(t, m.fny);
    ey = t - ez * m.ny;
}

__device__ __forceinline__ int64_t node_of(const hx::MeshView &m, int e, int i, int j, int k) {
    if (m.structured) {
        int ex, ey, ez;
        elem_xyz(m, e, ex, ey, ez);
        return (int64_t)(ex * HX_P + i) + m.Nx * ((int64_t)(ey * HX_P + j) + m.Ny * (int64_t)(ez * HX_P + k));
    }
    return m.dof_conn[(int64_t)e * NQ + i + N * (j + N * k)];
}

// EPB elements starting at e0 -> cubes (el*3 + c) of U; zero for padding
// elements and (if mask) constrained DoFs.
template <typename TV, typename T>
__device__ __forceinline__ void gather(const hx::MeshView &m, int e0, int epb, const TV *__restrict__ v, T *U,
                                       bool mask) {
    const int n = epb * NQ * 3;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
        const int c = idx % 3;
        const int a = (idx / 3) % NQ;
        const int el = idx / (3 * NQ);
        const int e = e0 + el;
        const int i = a % N, j = (a / N) % N, k = a / NN;
        T val = T(0);
        if (e < m.n_elem) {
            const int64_t d = 3 * node_of(m, e, i, j, k) + c;
            val = (T)v[d];
            if (mask && m.dmask && m.dmask[d]) val = T(0);
        }
        U[(el * 3 + c) * SZ + cidx(i, j, k)] = val;
    }
}

template <typename T>
__device__ __forceinline__ void scatter_add(const hx::MeshView &m, int e0, int epb, const T *U, T *__restrict__ out,
                                            bool mask) {
    const int n = epb * NQ * 3;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
        const int c = idx % 3;
        const int a = (idx / 3) % NQ;
        const int el = idx / (3 * NQ);
        const int e = e0 + el;
        if (e >= m.n_elem) continue;
        const int i = a % N, j = (a / N) % N, k = a / NN;
        if (m.elem_out) {  // ordered assembly: the gather pass sums and masks
            ((T *)m.elem_out)[3 * ((int64_t)e * NQ + a) + c] = U[(el * 3 + c) * SZ + cidx(i, j, k)];
            continue;
        }
        const int64_t d = 3 * node_of(m, e, i, j, k) + c;
        if (mask && m.dmask && m.dmask[d]) continue;
        atomicAdd(out + d, U[(el * 3 + c) * SZ + cidx(i, j, k)]);
    }
}

// ---------------------------------------------------------------------------
// small tensor algebra (row-major 3x3, sym6 = xx yy zz xy xz yz)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void mm(const T *A, const T *B, T *C) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) C[r * 3 + c] = fma(A[r * 3 + 0], B[0 * 3 + c], fma(A[r * 3 + 1], B[1 * 3 + c], A[r * 3 + 2] * B[2 * 3 + c]));
}

// 1/J-free inverse of F = I + Hk: adj(F) * invJ
template <typename T>
__device__ __forceinline__ void inv_F(const T *Hk, T invJ, T *Fi) {
    const T f00 = T(1) + Hk[0], f01 = Hk[1], f02 = Hk[2];
    const T f10 = Hk[3], f11 = T(1) + Hk[4], f12 = Hk[5];
    const T f20 = Hk[6], f21 = Hk[7], f22 = T(1) + Hk[8];
    Fi[0] = (f11 * f22 - f12 * f21) * invJ;
    Fi[1] = (f02 * f21 - f01 * f22) * invJ;
    Fi[2] = (f01 * f12 - f02 * f11) * invJ;
    Fi[3] = (f12 * f20 - f10 * f22) * invJ;
    Fi[4] = (f00 * f22 - f02 * f20) * invJ;
    Fi[5] = (f02 * f10 - f00 * f12) * invJ;
    Fi[6] = (f10 * f21 - f11 * f20) * invJ;
    Fi[7] = (f01 * f20 - f00 * f21) * invJ;
    Fi[8] = (f00 * f11 - f01 * f10) * invJ;
}

// J - 1 from the components of H = Grad u without forming det(I + H) - 1
// (Sec. "Stable and fast numerics"): det(I+H) - 1 = tr H + (tr^2 H - tr H^2)/2 + det H.
template <typename T>
__device__ __forceinline__ T J_minus_1(const T *H) {
    const T tr = H[0] + H[4] + H[8];
    const T tr2 = H[0] * H[0] + H[4] * H[4] + H[8] * H[8] + T(2) * (H[1] * H[3] + H[2] * H[6] + H[5] * H[7]);
    const T det = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                  H[2] * (H[3] * H[7] - H[4] * H[6]);
    return tr + T(0.5) * (tr * tr - tr2) + det;
}

// Green-Lagrange strain in stable form E = (H + H^T + H^T H)/2  (Eq. E_stable)
template <typename T>
__device__ __forceinline__ void green_strain(const T *H, T *E) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            T s = H[i * 3 + j] + H[j * 3 + i];
#pragma unroll
            for (int k = 0; k < 3; ++k) s = fma(H[k * 3 + i], H[k * 3 + j], s);
            E[SI(i, j)] = T(0.5) * s;
        }
}

// C^-1 = F^-1 F^-T (sym)
template <typename T>
__device__ __forceinline__ void cinv_from_Fi(const T *Fi, T *Ci) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j)
            Ci[SI(i, j)] = fma(Fi[i * 3 + 0], Fi[j * 3 + 0], fma(Fi[i * 3 + 1], Fi[j * 3 + 1], Fi[i * 3 + 2] * Fi[j * 3 + 2]));
}

// S = C^-1 (s1 E + s0 I) (the two factors commute; upper triangle kept)
template <typename T>
__device__ __forceinline__ void stress_CiX(const T *Ci, const T *E, T s1, T s0, T *S) {
    T X[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) X[k] = s1 * E[k];
    X[0] += s0;
    X[1] += s0;
    X[2] += s0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j)
            S[SI(i, j)] = fma(Ci[SI(i, 0)], X[SI(0, j)], fma(Ci[SI(i, 1)], X[SI(1, j)], Ci[SI(i, 2)] * X[SI(2, j)]));
}

// Alg. 2 (FastApproxJpow): J^-2/3 from J-1 by N_it Newton steps on x^-3 = J^2 from x0 = 1
template <typename T>
__device__ __forceinline__ T fast_jpow(T Jm1, int N_it) {
    const T alpha = ((Jm1 + T(2)) * Jm1 + T(1)) * T(1.0 / 3.0);
    T beta = T(4.0 / 3.0) - alpha;
    for (int n = 1; n < N_it; ++n) {
        const T b2 = beta * beta;
        beta = T(4.0 / 3.0) * beta - alpha * (b2 * b2);
    }
    return beta;
}

__device__ __forceinline__ double log1p_T(double x) { return log1p(x); }
__device__ __forceinline__ float log1p_T(float x) { return log1pf(x); }
__device__ __forceinline__ double exp_T(double x) { return exp(x); }
__device__ __forceinline__ float exp_T(float x) { return expf(x); }

// ---------------------------------------------------------------------------
// quadrature-point state of a law at Grad u_k = Hk (Sec. 4 stable forms)
// ---------------------------------------------------------------------------
template <typename T>
struct State {
    T Hk[9], Fi[9], Ci[6], S[6];
    T al, be, ga;       // D_uS = al sym(F^-1 H C^-1) + (be t + ga F:H) C^-1 + ga t I
    T ph4, ph6;         // fibre tangent factors c3 (2 k2 E_i^2 + 1) (0 if inactive)
    T H4[6], H6[6];     // structure tensors of the element
    // scalars kept by the cache-F strategy
    T invJ, lnJ, j23, c1, c2, s0, sg4, sg6;
    T Jm1;
};

// material constants in the compute precision (no per-point conversions)
template <typename T>
struct Mat {
    T mu, lambda, kappa, k1, k2;
};
template <typename T>
__device__ __forceinline__ Mat<T> mat_of(const hx::MeshView &m) {
    if constexpr (std::is_same<T, double>::value)
        return Mat<T>{m.mat.mu, m.mat.lambda, m.mat.kappa, m.mat.k1, m.mat.k2};
    else
        return Mat<T>{m.matf.mu, m.matf.lambda, m.matf.kappa, m.matf.k1, m.matf.k2};
}

template <typename T>
__device__ __forceinline__ void load_fibH(const hx::MeshView &m, int e, State<T> &st) {
    const T *fh = std::is_same<T, double>::value ? (const T *)m.fibH64 : (const T *)m.fibH;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        st.H4[k] = fh[(int64_t)k * m.n_elem + e];
        st.H6[k] = fh[(int64_t)(6 + k) * m.n_elem + e];
    }
}

// Full state from Hk, computed in T. FAST selects Alg. 2 for J^-2/3 (FP32
// on-the-fly paths); otherwise J^-2/3 = exp(-2/3 ln_{+1}(J-1)).
template <typename T, int LAW, bool FAST>
__device__ __forceinline__ void state_from_Hk(const hx::MeshView &m, int e, State<T> &st) {
    const Mat<T> mp = mat_of<T>(m);
    const T mu = mp.mu;
    st.Jm1 = J_minus_1(st.Hk);
    const T J = T(1) + st.Jm1;
    st.invJ = T(1) / J;
    inv_F(st.Hk, st.invJ, st.Fi);
    cinv_from_Fi(st.Fi, st.Ci);
    T E[6];
    green_strain(st.Hk, E);
    st.lnJ = log1p_T(st.Jm1);  // ln J = ln_{+1}(J - 1)
    if constexpr (LAW == HX_CNH) {
        const T lam = mp.lambda;
        stress_CiX(st.Ci, E, T(2) * mu, T(2) * lam * st.lnJ, st.S);
        st.al = T(2) * (mu - T(2) * lam * st.lnJ);
        st.be = T(2) * lam;
        st.ga = T(0);
        st.ph4 = st.ph6 = T(0);
    } else {
        const T kap = mp.kappa;
        st.j23 = FAST ? fast_jpow(st.Jm1, 3) : exp_T(T(-2.0 / 3.0) * st.lnJ);
        const T trE = E[0] + E[1] + E[2];
        const T vol = T(0.5) * kap * st.Jm1 * (st.Jm1 + T(2));  // kappa/2 (J^2 - 1), stable
        st.c1 = vol - mu * T(1.0 / 3.0) * st.j23 * (T(3) + T(2) * trE);
        st.c2 = mu * T(2.0 / 9.0) * st.j23 * (T(3) + T(2) * trE) + kap * J * J;
        st.s0 = vol - mu * T(2.0 / 3.0) * st.j23 * trE;
        stress_CiX(st.Ci, E, T(2) * mu * st.j23, st.s0, st.S);
        st.al = T(-2) * st.c1;
        st.be = st.c2;
        st.ga = mu * T(-2.0 / 3.0) * st.j23;
        st.ph4 = st.ph6 = T(0);
        st.sg4 = st.sg6 = T(0);
        if constexpr (LAW == HX_FIBER) {
            load_fibH(m, e, st);
            const T k1 = mp.k1, k2 = mp.k2;
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const T *Hf = f ? st.H6 : st.H4;
                // E_i = 2 H_i : E, I_i* - 1 = 2 M1.E.M1 (stable fibre invariants)
                T Ei = T(2) * (Hf[0] * E[0] + Hf[1] * E[1] + Hf[2] * E[2] +
                               T(2) * (Hf[3] * E[3] + Hf[4] * E[4] + Hf[5] * E[5]));
                T M[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) M[d] = (T)m.fibM[(int64_t)(3 * f + d) * m.n_elem + e];
                T mEm = M[0] * M[0] * E[0] + M[1] * M[1] * E[1] + M[2] * M[2] * E[2] +
                        T(2) * (M[0] * M[1] * E[3] + M[0] * M[2] * E[4] + M[1] * M[2] * E[5]);
                const T c3 = (mEm > T(0)) ? T(2) * k1 * exp_T(k2 * Ei * Ei) : T(0);
                const T sg = c3 * Ei, ph = c3 * (T(2) * k2 * Ei * Ei + T(1));
#pragma unroll
                for (int k = 0; k < 6; ++k) st.S[k] = fma(sg, Hf[k], st.S[k]);
                if (f) {
                    st.sg6 = sg;
                    st.ph6 = ph;
                } else {
                    st.sg4 = sg;
                    st.ph4 = ph;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// cache layouts (SoA [field][n_qp])
//  cache-F:      0-8 Hk, 9 1/J, then cNH: 10 ln J
//                iNH/fiber: 10 J^-2/3, 11 c1, 12 c2, 13 s0 (stress scalar);
//                fiber: 14 sigma_4, 15 sigma_6, 16 phi_4, 17 phi_6
//  cache-tensors: 0-8 Hk, 9-17 F^-1, 18-23 C^-1, 24-29 S, 30 alpha,
//                iNH/fiber: 31 beta, 32 gamma; fiber: 33 phi_4, 34 phi_6
// ---------------------------------------------------------------------------
template <typename TS, int LAW, int STORAGE>
__device__ __forceinline__ void store_state(TS *qp, int64_t nq, int64_t g, const State<double> &st) {
    auto put = [&](int f, double v) { qp[(int64_t)f * nq + g] = (TS)v; };
#pragma unroll
    for (int k = 0; k < 9; ++k) put(k, st.Hk[k]);
    if constexpr (STORAGE == HX_CACHE_F) {
        put(9, st.invJ);
        if constexpr (LAW == HX_CNH) {
            put(10, st.lnJ);
        } else {
            put(10, st.j23);
            put(11, st.c1);
            put(12, st.c2);
            put(13, st.s0);
            if constexpr (LAW == HX_FIBER) {
                put(14, st.sg4);
                put(15, st.sg6);
                put(16, st.ph4);
                put(17, st.ph6);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) put(9 + k, st.Fi[k]);
#pragma unroll
        for (int k = 0; k < 6; ++k) put(18 + k, st.Ci[k]);
#pragma unroll
        for (int k = 0; k < 6; ++k) put(24 + k, st.S[k]);
        put(30, st.al);
        if constexpr (LAW != HX_CNH) {
            put(31, st.be);
            put(32, st.ga);
            if constexpr (LAW == HX_FIBER) {
                put(33, st.ph4);
                put(34, st.ph6);
            }
        }
    }
}

// state of the cache strategies from the stored fields; get(f) returns field f
template <typename T, int LAW, int STORAGE, typename Get>
__device__ __forceinline__ void build_state(const hx::MeshView &m, int e, Get get, State<T> &st) {
    const Mat<T> mp = mat_of<T>(m);
    const T mu = mp.mu;
#pragma unroll
    for (int k = 0; k < 9; ++k) st.Hk[k] = get(k);
    st.ph4 = st.ph6 = T(0);
    if constexpr (STORAGE == HX_CACHE_F) {
        st.invJ = get(9);
        inv_F(st.Hk, st.invJ, st.Fi);
        cinv_from_Fi(st.Fi, st.Ci);
        T E[6];
        green_strain(st.Hk, E);
        if constexpr (LAW == HX_CNH) {
            const T lam = mp.lambda;
            const T lnJ = get(10);
            stress_CiX(st.Ci, E, T(2) * mu, T(2) * lam * lnJ, st.S);
            st.al = T(2) * (mu - T(2) * lam * lnJ);
            st.be = T(2) * lam;
            st.ga = T(0);
        } else {
            const T j23 = get(10);
            st.c1 = get(11);
            st.c2 = get(12);
            const T s0 = get(13);
            stress_CiX(st.Ci, E, T(2) * mu * j23, s0, st.S);
            st.al = T(-2) * st.c1;
            st.be = st.c2;
            st.ga = mu * T(-2.0 / 3.0) * j23;
            if constexpr (LAW == HX_FIBER) {
                load_fibH(m, e, st);
                const T sg4 = get(14), sg6 = get(15);
#pragma unroll
                for (int k = 0; k < 6; ++k) st.S[k] = fma(sg4, st.H4[k], fma(sg6, st.H6[k], st.S[k]));
                st.ph4 = get(16);
                st.ph6 = get(17);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) st.Fi[k] = get(9 + k);
#pragma unroll
        for (int k = 0; k < 6; ++k) st.Ci[k] = get(18 + k);
#pragma unroll
        for (int k = 0; k < 6; ++k) st.S[k] = get(24 + k);
        st.al = get(30);
        if constexpr (LAW == HX_CNH) {
            st.be = T(2) * mp.lambda;
            st.ga = T(0);
        } else {
            st.be = get(31);
            st.ga = get(32);
            if constexpr (LAW == HX_FIBER) {
                load_fibH(m, e, st);
                st.ph4 = get(33);
                st.ph6 = get(34);
            }
        }
    }
}

template <typename T, int LAW, int STORAGE>
__device__ __forceinline__ void load_state(const hx::MeshView &m, int e, int64_t g, State<T> &st) {
    const T *qp = (const T *)m.qp;
    const int64_t nq = m.qs;
    build_state<T, LAW, STORAGE>(m, e, [&](int f) { return __ldcs(qp + (int64_t)f * nq + g); }, st);
}

// dP = H S + F D_uS[H] for a physical displacement-gradient direction H
// (Sec. 2 Eq. DDu_residual_material; D_uS from App. A with the sign of the
// D_uC^-1 term that follows from differentiating S).
template <typename T, int LAW>
__device__ __forceinline__ void tangent_dP(const State<T> &st, const T *H, T *dP) {
    T A[9];
    mm(st.Fi, H, A);  // F^-1 H
    const T t = A[0] + A[4] + A[8];
    T D[6];
    // sym(F^-1 H C^-1)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            const T bij = fma(A[i * 3 + 0], st.Ci[SI(0, j)], fma(A[i * 3 + 1], st.Ci[SI(1, j)], A[i * 3 + 2] * st.Ci[SI(2, j)]));
            const T bji = fma(A[j * 3 + 0], st.Ci[SI(0, i)], fma(A[j * 3 + 1], st.Ci[SI(1, i)], A[j * 3 + 2] * st.Ci[SI(2, i)]));
            D[SI(i, j)] = T(0.5) * st.al * (bij + bji);
        }
    T cC = st.be * t;
    if constexpr (LAW != HX_CNH) {
        T FH = H[0] + H[4] + H[8];  // F : H = tr H + Hk : H
#pragma unroll
        for (int k = 0; k < 9; ++k) FH = fma(st.Hk[k], H[k], FH);
        cC = fma(st.ga, FH, cC);
        const T gt = st.ga * t;
        D[0] += gt;
        D[1] += gt;
        D[2] += gt;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) D[k] = fma(cC, st.Ci[k], D[k]);
    if constexpr (LAW == HX_FIBER) {
        // H_i : D_uC with D_uC = 2 sym(F^T H), F^T H = H + Hk^T H
        T FtH[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                FtH[i * 3 + j] = H[i * 3 + j] + fma(st.Hk[0 * 3 + i], H[0 * 3 + j], fma(st.Hk[1 * 3 + i], H[1 * 3 + j], st.Hk[2 * 3 + i] * H[2 * 3 + j]));
        auto contract = [&](const T *Hs) {
            return T(2) * (Hs[0] * FtH[0] + Hs[1] * FtH[4] + Hs[2] * FtH[8] + Hs[3] * (FtH[1] + FtH[3]) +
                           Hs[4] * (FtH[2] + FtH[6]) + Hs[5] * (FtH[5] + FtH[7]));
        };
        const T f4 = st.ph4 * contract(st.H4);
        const T f6 = st.ph6 * contract(st.H6);
#pragma unroll
        for (int k = 0; k < 6; ++k) D[k] = fma(f4, st.H4[k], fma(f6, st.H6[k], D[k]));
    }
    // dP = H S + D + Hk D
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            T s = D[SI(c, d)];
#pragma unroll
            for (int k = 0; k < 3; ++k) s = fma(H[c * 3 + k], st.S[SI(k, d)], fma(st.Hk[c * 3 + k], D[SI(k, d)], s));
            dP[c * 3 + d] = s;
        }
}

template <typename T>
__device__ __forceinline__ void load_geo(const hx::MeshView &m, int64_t g, T *Ji, T &JxW) {
    const T *geo = (const T *)m.geo;
#pragma unroll
    for (int k = 0; k < 9; ++k) Ji[k] = __ldcs(geo + (int64_t)k * m.qs + g);
    JxW = __ldcs(geo + (int64_t)9 * m.qs + g);
}

// physical gradient H = G J0^-1 from the reference gradient G (G_{cd} = du_c/dxi_d)
template <typename T>
__device__ __forceinline__ void push_grad(const T *G, const T *Ji, T *H) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d) H[c * 3 + d] = fma(G[c * 3 + 0], Ji[0 * 3 + d], fma(G[c * 3 + 1], Ji[1 * 3 + d], G[c * 3 + 2] * Ji[2 * 3 + d]));
}

// test-side pull back Q = JxW P J0^-T (Q_{ce} = JxW sum_d P_cd (J0^-1)_{ed})
template <typename T>
__device__ __forceinline__ void pull_flux(const T *P, const T *Ji, T JxW, T *Q) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int e = 0; e < 3; ++e) Q[c * 3 + e] = JxW * fma(P[c * 3 + 0], Ji[e * 3 + 0], fma(P[c * 3 + 1], Ji[e * 3 + 1], P[c * 3 + 2] * Ji[e * 3 + 2]));
}

// ---------------------------------------------------------------------------
// Integration over the spatial configuration (Sec. 2, Eq.
// stress_term_in_Ot_with_JC; Sec. 5 "spatial integration" paragraphs). With
// g = grad du = (Grad du) F^-1 = G J_t^-1 (J_t = F J0, the deformed mapping)
// the tangent integrand is (grad v) : [Jc:g^S + g tau] over Omega_0, i.e.
//   Q = JxW (Jc:g^S + g tau) J_t^-T.
// Per law (c1, c2 of Sec. 5; b = F F^T; h_i = F H_i F^T; j = J^-2/3; the iNH
// moduli pushed forward from the material D_uS, whose I (x) C^-1 part gives
// tr(e) b + (b:e) I):
//   cNH:   tau = mu b - c I,  Jc:e = 2c e + 2 lambda tr(e) I,  c = mu - 2 lambda ln J
//   iNH:   tau = mu j b + c1 I,
//          Jc:e = -2 c1 e + c2 tr(e) I - (2 mu/3) j [tr(e) b + (b:e) I]
//   fiber: tau += sum_i c3 E_i h_i,  Jc:e += sum_i 2 c3 (2 k2 E_i^2 + 1) (h_i:e) h_i
// The multiples of g from the I-part of tau cancel against those of Jc:g^S,
// which leaves
//   sigma = g T + a g^T + (b tr g + B:g) I + tr(g) B + sum_i (h^_i:g) h^_i
// with T = mu b (cNH) or mu j b + sum_i c3 E_i h_i, a = c (cNH) or -c1,
// b = 2 lambda (cNH) or c2, B = -(2 mu/3) j b (iNH, fiber) and
// h^_i = sqrt(2 c3 (2 k2 E_i^2 + 1)) h_i. Every stored tensor and scalar is
// multiplied by JxW (h^_i by its square root), so that Q = sigma J_t^-T.
// Field layout (SoA [field][n_qp]): 0-8 J_t^-1 (row-major, g = G J_t^-1),
// 9-14 T (sym6), 15 a, 16 b; iNH/fiber 17-22 B (sym6); fiber 23-28 h^_4,
// 29-34 h^_6.
// ---------------------------------------------------------------------------
template <int LAW>
__device__ __forceinline__ void spatial_fields(const State<double> &st, const double *Ji, double JxW,
                                               const hx::MeshView &m, double *f) {
    const double mu = m.mat.mu;
    // J_t^-1 = J0^-1 F^-1
#pragma unroll
    for (int e = 0; e < 3; ++e)
#pragma unroll
        for (int d = 0; d < 3; ++d)
            f[e * 3 + d] = Ji[e * 3 + 0] * st.Fi[0 * 3 + d] + Ji[e * 3 + 1] * st.Fi[1 * 3 + d] + Ji[e * 3 + 2] * st.Fi[2 * 3 + d];
    // b = F F^T = I + Hk + Hk^T + Hk Hk^T (no I - I cancellation in the strain part)
    double b[6];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            double v = st.Hk[i * 3 + j] + st.Hk[j * 3 + i];
#pragma unroll
            for (int k = 0; k < 3; ++k) v += st.Hk[i * 3 + k] * st.Hk[j * 3 + k];
            b[SI(i, j)] = v + (i == j ? 1.0 : 0.0);
        }
    double T[6], a, bb;
    if constexpr (LAW == HX_CNH) {
#pragma unroll
        for (int k = 0; k < 6; ++k) T[k] = mu * b[k];
        a = mu - 2.0 * m.mat.lambda * st.lnJ;
        bb = 2.0 * m.mat.lambda;
    } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) T[k] = mu * st.j23 * b[k];
        a = -st.c1;
        bb = st.c2;
        const double ga = -(2.0 / 3.0) * mu * st.j23;
#pragma unroll
        for (int k = 0; k < 6; ++k) f[17 + k] = JxW * ga * b[k];
        if constexpr (LAW == HX_FIBER) {
            double F[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) F[k] = st.Hk[k] + ((k % 4) == 0 ? 1.0 : 0.0);
#pragma unroll
            for (int fam = 0; fam < 2; ++fam) {
                const double *Hs = fam ? st.H6 : st.H4;
                // h = F H_i F^T
                double FH[9];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        FH[i * 3 + j] = F[i * 3 + 0] * Hs[SI(0, j)] + F[i * 3 + 1] * Hs[SI(1, j)] + F[i * 3 + 2] * Hs[SI(2, j)];
                double h[6];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = i; j < 3; ++j)
                        h[SI(i, j)] = FH[i * 3 + 0] * F[j * 3 + 0] + FH[i * 3 + 1] * F[j * 3 + 1] + FH[i * 3 + 2] * F[j * 3 + 2];
                const double sg = fam ? st.sg6 : st.sg4;   // c3 E_i
                const double ph = fam ? st.ph6 : st.ph4;   // c3 (2 k2 E_i^2 + 1) >= 0
                const double sc = sqrt(JxW * 2.0 * ph);
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    T[k] += sg * h[k];
                    f[23 + 6 * fam + k] = sc * h[k];
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) f[9 + k] = JxW * T[k];
    f[15] = JxW * a;
    f[16] = JxW * bb;
}

// Q = sigma(g) J_t^-T from the reference gradient G and the stored fields
// (get(f) returns field f)
template <typename T, int LAW, typename Get>
__device__ __forceinline__ void spatial_Q(const T *G, Get get, T *Q) {
    T Jt[9], g[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Jt[k] = get(k);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d) g[c * 3 + d] = fma(G[c * 3 + 0], Jt[0 * 3 + d], fma(G[c * 3 + 1], Jt[1 * 3 + d], G[c * 3 + 2] * Jt[2 * 3 + d]));
    const T tr = g[0] + g[4] + g[8];
    T Ts[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) Ts[k] = get(9 + k);
    const T a = get(15);
    T diag = get(16) * tr;
    T sig[9];
    if constexpr (LAW != HX_CNH) {
        T Bs[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) Bs[k] = get(17 + k);
        diag = fma(Bs[0], g[0], fma(Bs[1], g[4], fma(Bs[2], g[8], diag)));
        diag = fma(Bs[3], g[1] + g[3], fma(Bs[4], g[2] + g[6], fma(Bs[5], g[5] + g[7], diag)));
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) sig[c * 3 + d] = tr * Bs[SI(c, d)];
    } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) sig[k] = T(0);
    }
    if constexpr (LAW == HX_FIBER) {
#pragma unroll
        for (int fam = 0; fam < 2; ++fam) {
            T h[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) h[k] = get(23 + 6 * fam + k);
            T hg = h[0] * g[0];
            hg = fma(h[1], g[4], fma(h[2], g[8], hg));
            hg = fma(h[3], g[1] + g[3], fma(h[4], g[2] + g[6], fma(h[5], g[5] + g[7], hg)));
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int d = 0; d < 3; ++d) sig[c * 3 + d] = fma(hg, h[SI(c, d)], sig[c * 3 + d]);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            T s = fma(a, g[d * 3 + c], sig[c * 3 + d]);
            if (c == d) s += diag;
            s = fma(g[c * 3 + 0], Ts[SI(0, d)], fma(g[c * 3 + 1], Ts[SI(1, d)], fma(g[c * 3 + 2], Ts[SI(2, d)], s)));
            sig[c * 3 + d] = s;
        }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int e = 0; e < 3; ++e) Q[c * 3 + e] = fma(sig[c * 3 + 0], Jt[e * 3 + 0], fma(sig[c * 3 + 1], Jt[e * 3 + 1], sig[c * 3 + 2] * Jt[e * 3 + 2]));
}

__device__ __forceinline__ void flag_state(const hx::MeshView &m, double Jm1) {
    if (!(Jm1 > -1.0)) {
        if (Jm1 != Jm1)
            atomicOr(m.err + 1, 1);
        else
            atomicOr(m.err + 0, 1);
    }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// column-layout building blocks of the apply kernel: every element has n^2
// threads; thread (a0, a1) owns one line of each direction (x-line (j,k) =
// (a0,a1), y-line (i,k), z-line (i,j)), and the z-line also carries the
// quadrature-point column (a0, a1, *) through the material phase in registers
// ---------------------------------------------------------------------------
template <int DIR>
__device__ __forceinline__ int line_off(int a0, int a1) {
    if constexpr (DIR == 0) return a0 * CRS + a1 * CPS;
    else if constexpr (DIR == 1) return a0 + a1 * CPS;
    else return a0 + a1 * CRS;
}
template <int DIR>
__device__ __forceinline__ constexpr int line_str() {
    return DIR == 0 ? 1 : (DIR == 1 ? CRS : CPS);
}
template <int DIR>
__device__ __forceinline__ void ld_line(const Real *p, Real *x) {
#pragma unroll
    for (int t = 0; t < N; ++t) x[t] = p[t * line_str<DIR>()];
}
template <int DIR>
__device__ __forceinline__ void st_line(Real *p, const Real *y) {
#pragma unroll
    for (int t = 0; t < N; ++t) p[t * line_str<DIR>()] = y[t];
}
// y = M x (TR: y = M^T x) with a 1D table from constant memory. With EO and
// from five points on, the even-odd decomposition: with e_t = x_t + x_{N-1-t}
// and d_t = x_t - x_{N-1-t}, a_o = P e (+ M[o][h] x_h), b_o = Q d,
// y_o = a_o + b_o and y_{N-1-o} = +-(a_o - b_o) (N^2 FMAs become about
// N^2/2 + 2N). FP64 units use it everywhere (their apply is bound by the FP64
// pipe); FP32 units only in the staged apply, which is bound by instruction
// issue. The FP32 residual and register-path sweeps keep the plain products:
// a_o - b_o loses relative accuracy where the two nearly cancel, which took
// the FP32 residual at p = 6 past a relative error of 1e-5.
template <int TAB, bool TR, bool EO = (sizeof(Real) == 8)>
__device__ __forceinline__ void mv(const Real *x, Real *y) {
    if constexpr (N >= 5 && EO) {
        constexpr int H = EOH;
        constexpr bool SYM = TAB == TB;
        auto M = [](int o, int t) { return tab<TAB>(TR ? t * N + o : o * N + t); };
        Real ev[H], od[H];
#pragma unroll
        for (int t = 0; t < H; ++t) {
            ev[t] = x[t] + x[N - 1 - t];
            od[t] = x[t] - x[N - 1 - t];
        }
#pragma unroll
        for (int o = 0; o < H; ++o) {
            Real a = Real(0), b = Real(0);
#pragma unroll
            for (int t = 0; t < H; ++t) {
                a = fma(cEO[TAB][TR][0][o * H + t], ev[t], a);
                b = fma(cEO[TAB][TR][1][o * H + t], od[t], b);
            }
            if constexpr (N % 2 == 1) a = fma(M(o, H), x[H], a);
            y[o] = a + b;
            y[N - 1 - o] = SYM ? a - b : b - a;
        }
        if constexpr (N % 2 == 1) {
            Real c = Real(0);
#pragma unroll
            for (int t = 0; t < H; ++t) c = fma(M(H, t), SYM ? ev[t] : od[t], c);
            if constexpr (SYM) c = fma(M(H, H), x[H], c);
            y[H] = c;
        }
    } else {
#pragma unroll
        for (int o = 0; o < N; ++o) {
            Real s = Real(0);
#pragma unroll
            for (int t = 0; t < N; ++t) s = fma(tab<TAB>(TR ? t * N + o : o * N + t), x[t], s);
            y[o] = s;
        }
    }
}

// Paired sweeps (FP32 units): two independent lines through one 1D table at
// once with the packed FP32 instructions of sm_100 and later (FFMA2, one
// instruction per two products). Each lane performs mv's operations in mv's
// order, so the results are those of two mv calls. The tables are read as
// {m, m} pairs from cTab2 and cEO2 (copies of cTab and cEO).
__constant__ float2 cTab2[3][NN];
__constant__ float2 cEO2[3][2][2][(EOH > 0 ? EOH : 1) * (EOH > 0 ? EOH : 1)];
constexpr bool PK = sizeof(Real) == 4;

__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

template <int TAB, bool TR, bool EO>
__device__ __forceinline__ void mv2(const float2 *x, float2 *y) {
    auto M = [](int o, int t) { return cTab2[TAB][TR ? t * N + o : o * N + t]; };
    if constexpr (N >= 5 && EO) {
        constexpr int H = EOH;
        constexpr bool SYM = TAB == TB;
        float2 ev[H], od[H];
#pragma unroll
        for (int t = 0; t < H; ++t) {
            ev[t] = __fadd2_rn(x[t], x[N - 1 - t]);
            od[t] = sub2(x[t], x[N - 1 - t]);
        }
#pragma unroll
        for (int o = 0; o < H; ++o) {
            float2 a = __fmul2_rn(cEO2[TAB][TR][0][o * H], ev[0]);
            float2 b = __fmul2_rn(cEO2[TAB][TR][1][o * H], od[0]);
#pragma unroll
            for (int t = 1; t < H; ++t) {
                a = __ffma2_rn(cEO2[TAB][TR][0][o * H + t], ev[t], a);
                b = __ffma2_rn(cEO2[TAB][TR][1][o * H + t], od[t], b);
            }
            if constexpr (N % 2 == 1) a = __ffma2_rn(M(o, H), x[H], a);
            y[o] = __fadd2_rn(a, b);
            y[N - 1 - o] = SYM ? sub2(a, b) : sub2(b, a);
        }
        if constexpr (N % 2 == 1) {
            float2 c = __fmul2_rn(M(H, 0), SYM ? ev[0] : od[0]);
#pragma unroll
            for (int t = 1; t < H; ++t) c = __ffma2_rn(M(H, t), SYM ? ev[t] : od[t], c);
            if constexpr (SYM) c = __ffma2_rn(M(H, H), x[H], c);
            y[H] = c;
        }
    } else {
#pragma unroll
        for (int o = 0; o < N; ++o) {
            float2 s = __fmul2_rn(M(o, 0), x[0]);
#pragma unroll
            for (int t = 1; t < N; ++t) s = __ffma2_rn(M(o, t), x[t], s);
            y[o] = s;
        }
    }
}
// y_c = M x_c for the three components of a thread's lines: components 0 and
// 1 paired, component 2 alone in FP32 units; three mv calls otherwise
template <int TAB, bool TR, bool EO>
__device__ __forceinline__ void mv3(const Real (*x)[N], Real (*y)[N]) {
    if constexpr (PK) {
        float2 a[N], b[N];
#pragma unroll
        for (int t = 0; t < N; ++t) a[t] = make_float2(x[0][t], x[1][t]);
        mv2<TAB, TR, EO>(a, b);
#pragma unroll
        for (int t = 0; t < N; ++t) {
            y[0][t] = b[t].x;
            y[1][t] = b[t].y;
        }
        mv<TAB, TR, EO>(x[2], y[2]);
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) mv<TAB, TR, EO>(x[c], y[c]);
    }
}
// y_c = M x_c and v_c = M u_c (six independent lines): three pairs in FP32
// units, six mv calls otherwise
template <int TAB, bool TR, bool EO>
__device__ __forceinline__ void mv6(const Real (*x)[N], const Real (*u)[N], Real (*y)[N], Real (*v)[N]) {
    if constexpr (PK) {
        float2 a[3][N], b[3][N];
#pragma unroll
        for (int t = 0; t < N; ++t) {
            a[0][t] = make_float2(x[0][t], x[1][t]);
            a[1][t] = make_float2(x[2][t], u[0][t]);
            a[2][t] = make_float2(u[1][t], u[2][t]);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) mv2<TAB, TR, EO>(a[k], b[k]);
#pragma unroll
        for (int t = 0; t < N; ++t) {
            y[0][t] = b[0][t].x;
            y[1][t] = b[0][t].y;
            y[2][t] = b[1][t].x;
            v[0][t] = b[1][t].y;
            v[1][t] = b[2][t].x;
            v[2][t] = b[2][t].y;
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            mv<TAB, TR, EO>(x[c], y[c]);
            mv<TAB, TR, EO>(u[c], v[c]);
        }
    }
}

// Two FP32 values computed lane-wise with the packed FP32 instructions
// (FFMA2, FADD2, FMUL2): each lane performs the scalar operation with one
// rounding, so a function templated on its scalar type gives, per lane, the
// scalar function's result.
struct F2 {
    float2 v;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ F2(int z) : v(make_float2((float)z, (float)z)) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
    // hidden friends: found for F2 arguments only, so that the scalar fma and
    // operators keep their meaning everywhere else
    __device__ __forceinline__ friend F2 operator+(F2 a, F2 b) {
        F2 r;
        r.v = __fadd2_rn(a.v, b.v);
        return r;
    }
    __device__ __forceinline__ friend F2 operator*(F2 a, F2 b) {
        F2 r;
        r.v = __fmul2_rn(a.v, b.v);
        return r;
    }
    __device__ __forceinline__ friend F2 &operator+=(F2 &a, F2 b) {
        a.v = __fadd2_rn(a.v, b.v);
        return a;
    }
    __device__ __forceinline__ friend F2 fma(F2 a, F2 b, F2 c) {
        F2 r;
        r.v = __ffma2_rn(a.v, b.v, c.v);
        return r;
    }
};

// node numbering base of an element (structured box: lattice index of its
// first node; otherwise the element index for the connectivity lookup)
__device__ __forceinline__ int64_t elem_base(const hx::MeshView &m, int e) {
    if (e >= m.n_elem) return 0;
    if (m.structured) {
        int ex, ey, ez;
        elem_xyz(m, e, ex, ey, ez);
        return (int64_t)ex * HX_P + m.Nx * ((int64_t)ey * HX_P + m.Ny * (int64_t)ez * HX_P);
    }
    return e;
}
__device__ __forceinline__ int64_t node_at(const hx::MeshView &m, int64_t base, int i, int j, int k) {
    if (m.structured) return base + i + m.Nx * (j + m.Ny * (int64_t)k);
    return m.dof_conn[base * NQ + i + N * (j + N * k)];
}

// L2 cache policies: the quadrature-point stream is read once per apply
// (evict first); the DoF vectors are gathered and scattered by up to eight
// elements each and should stay resident (evict last)
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes, uint64_t pol) {
    asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(p), "r"(bytes), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ float ld_stream(const float *p, uint64_t pol) {
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_stream(const double *p, uint64_t pol) {
    double v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void red_add(float *p, float v, uint64_t pol) {
    asm volatile("red.global.add.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void red_add(double *p, double v, uint64_t pol) {
    asm volatile("red.global.add.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
}


// Load the x-row (j = a0, k = a1) of element e of vector v into registers:
// row[3*i + c] = v_c at node (i, a0, a1). In a structured box the row is 3*N
// contiguous values; otherwise the N node ids come from the connectivity.
// Constrained DoFs (mask) and elements past the end read zero.
__device__ __forceinline__ void load_row(const hx::MeshView &m, int e, int64_t base, int a0, int a1,
                                         const Real *__restrict__ v, bool mask, Real *row) {
    if (e >= m.n_elem) {
#pragma unroll
        for (int t = 0; t < 3 * N; ++t) row[t] = Real(0);
        return;
    }
    if (m.structured) {
        const int64_t off = 3 * (base + m.Nx * (a0 + m.Ny * (int64_t)a1));
        const Real *p = v + off;
#pragma unroll
        for (int t = 0; t < 3 * N; ++t) row[t] = p[t];
        if (mask && m.dmask) {
            const uint8_t *q = m.dmask + off;
#pragma unroll
            for (int t = 0; t < 3 * N; ++t)
                if (q[t]) row[t] = Real(0);
        }
    } else {
        const int32_t *cn = m.dof_conn + (int64_t)e * NQ + N * (a0 + N * a1);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const int64_t d = 3 * (int64_t)cn[i];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                row[3 * i + c] = v[d + c];
                if (mask && m.dmask && m.dmask[d + c]) row[3 * i + c] = Real(0);
            }
        }
    }
}

// Subtract from a thread's x-row of v (3 N values, load_row layout) the value
// of v at its element's node (0, 0, 0). For rows of a field whose gradient is
// all that is needed (u in the residual, u_k in the recompute strategy): a
// smooth field's nodal values are about |v| / h times its gradient, and
// differentiating them directly in FP32 would lose that factor to
// cancellation; the gradient of the shifted rows is the same.
__device__ __forceinline__ void shift_row(const hx::MeshView &m, int e, int64_t base, const Real *__restrict__ v,
                                          Real *row) {
    if (e >= m.n_elem) return;
    const int64_t d = 3 * node_at(m, base, 0, 0, 0);
    const Real s0 = v[d], s1 = v[d + 1], s2 = v[d + 2];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        row[3 * i + 0] -= s0;
        row[3 * i + 1] -= s1;
        row[3 * i + 2] -= s2;
    }
}

// forward sum factorization of an element whose x-rows are in the threads'
// registers (row[3*i + c], x-line (a0, a1)): leaves the x-, y- and
// z-reference derivatives at the Gauss points in X0, X1 and X2, which also
// serve as scratch. X0 must not be read by other threads when the call starts
// (the last phase of the previous tile reads X1 only); the caller places a
// CTA barrier after the call before the derivatives are read.
__device__ __forceinline__ void col_forward(const Real *row, Real *X0, Real *X1, Real *X2, bool act, int eoff, int a0,
                                            int a1) {
    Real x[N], y[N];
    const int o0 = eoff + line_off<0>(a0, a1), o1 = eoff + line_off<1>(a0, a1), o2 = eoff + line_off<2>(a0, a1);
    if (act) {  // x-lines: X0 = Bx u
#pragma unroll
        for (int c = 0; c < 3; ++c) {
#pragma unroll
            for (int i = 0; i < N; ++i) x[i] = row[3 * i + c];
            mv<TB, false>(x, y);
            st_line<0>(X0 + c * CCZ + o0, y);
        }
    }
    __syncthreads();
    if (act) {  // y-lines: X1 = By X0
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ld_line<1>(X0 + c * CCZ + o1, x);
            mv<TB, false>(x, y);
            st_line<1>(X1 + c * CCZ + o1, y);
        }
    }
    __syncthreads();
    if (act) {  // z-lines: values V = Bz X1 (in place, per line) and X2 = Dz V
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ld_line<2>(X1 + c * CCZ + o2, x);
            mv<TB, false>(x, y);
            st_line<2>(X1 + c * CCZ + o2, y);
            mv<TD, false>(y, x);
            st_line<2>(X2 + c * CCZ + o2, x);
        }
    }
    __syncthreads();
    Real dy[3][N];
    if (act) {  // x-lines: X0 = Dx V (X0 is free); y-lines: Dy V held until V is read
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ld_line<0>(X1 + c * CCZ + o0, x);
            mv<TD, false>(x, y);
            st_line<0>(X0 + c * CCZ + o0, y);
            ld_line<1>(X1 + c * CCZ + o1, x);
            mv<TD, false>(x, dy[c]);
        }
    }
    __syncthreads();  // every y-line of V has been read
    if (act) {
#pragma unroll
        for (int c = 0; c < 3; ++c) st_line<1>(X1 + c * CCZ + o1, dy[c]);
    }
}

// Barrier between the phases of a tile: the whole CTA, or (WS) the warp alone
// when every element's cubes and stage belong to one warp.
template <bool WS>
__device__ __forceinline__ void phase_sync() {
    if constexpr (WS)
        __syncwarp();
    else
        __syncthreads();
}

// Forward sweeps for the column-ordered quadrature-point phase: as
// col_forward, but the z-derivative of each thread's z-line (its column of
// quadrature points, (qx, qy) = (a0, a1)) stays in registers gz[c][k], the
// x-derivative goes to X0 and the y-derivative to X2 (X1 keeps the values).
// No final barrier (the caller's barrier completes the sweeps).
template <bool SW, bool WS = false>
__device__ __forceinline__ void col_forward_c(const Real *row, Real *X0, Real *X1, Real *X2, Real (*gz)[N], bool act,
                                              int eoff, const LineOffs<SW> &o) {
    // each phase loads all three components' lines before any store: the
    // cubes share one allocation, so the compiler may not move a load above
    // a store itself
    constexpr int CZ = Lay<SW>::CZ;
    constexpr bool EO = true;  // even-odd sweeps in the staged apply (see mv)
    Real x[3][N], y[3][N];
    if (act) {  // x-lines: X0 = Bx u
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < N; ++i) x[c][i] = row[3 * i + c];
        mv3<TB, false, EO>(x, y);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < N; ++i) X0[eoff + c * CZ + o.x + i] = y[c][i];
    }
    phase_sync<WS>();
    if (act) {  // y-lines: X1 = By X0
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int t = 0; t < N; ++t) x[c][t] = X0[eoff + c * CZ + o.y[t]];
        mv3<TB, false, EO>(x, y);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int t = 0; t < N; ++t) X1[eoff + c * CZ + o.y[t]] = y[c][t];
    }
    phase_sync<WS>();
    if (act) {  // z-lines: values V = Bz X1 (in place, per line), Dz V kept
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int t = 0; t < N; ++t) x[c][t] = X1[eoff + c * CZ + o.z[t]];
        mv3<TB, false, EO>(x, y);
        mv3<TD, false, EO>(y, gz);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int t = 0; t < N; ++t) X1[eoff + c * CZ + o.z[t]] = y[c][t];
    }
    phase_sync<WS>();
    if (act) {  // x-lines: X0 = Dx V; y-lines: X2 = Dy V
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int t = 0; t < N; ++t) {
                x[c][t] = X1[eoff + c * CZ + o.x + t];
                y[c][t] = X1[eoff + c * CZ + o.y[t]];
            }
        Real dx[3][N], dy[3][N];
        mv6<TD, false, EO>(x, y, dx, dy);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int t = 0; t < N; ++t) {
                X0[eoff + c * CZ + o.x + t] = dx[c][t];
                X2[eoff + c * CZ + o.y[t]] = dy[c][t];
            }
    }
}

// L2 prefetch of a tile's quadrature-point data (geometry + cache), one
// contiguous chunk per field; skipped where a chunk is not 16-byte aligned
template <int EPB, int STORAGE>
__device__ __forceinline__ void prefetch_tile(const hx::MeshView &m, int tile) {
    const int e0 = tile * EPB;
    if (e0 >= m.n_elem) return;
    const int cnt = min(EPB, m.n_elem - e0);
    const unsigned bytes = (unsigned)(cnt * NQ * sizeof(Real));
    const int nfc = STORAGE == HX_RECOMPUTE ? 0 : m.nf;
    constexpr int ng = STORAGE == HX_SPATIAL_TENSORS ? 0 : 10;
    const int f = threadIdx.x;
    if (f >= ng + nfc || (bytes & 15u)) return;
    const Real *p = f < ng ? (const Real *)m.geo + (int64_t)f * m.qs + (int64_t)e0 * NQ
                           : (const Real *)m.qp + (int64_t)(f - ng) * m.qs + (int64_t)e0 * NQ;
    if (((uintptr_t)p & 15u) == 0) prefetch_l2(p, bytes, policy_evict_first());
}

// quadrature-point fields a strategy reads per point: geometry (J0^-1, JxW;
// not for the spatial strategy, whose fields carry J_t^-1) and the cache
template <int LAW, int STORAGE>
struct QpFields {
    static constexpr int ng = STORAGE == HX_SPATIAL_TENSORS ? 0 : 10;
    static constexpr int nc = STORAGE == HX_RECOMPUTE ? 0 : hx::qp_fields(LAW, STORAGE);
    static constexpr int n = ng + nc;
};

// Shared memory of an apply CTA: three cubes per element (six for the
// recompute strategy, which also interpolates Grad u_k), then, for the staged
// variant, the tile's quadrature-point fields (one EPB*NQ chunk per field).
template <int EPB, int LAW, int STORAGE, bool STAGED>
struct ApplySmem {
    static constexpr int arrays = STORAGE == HX_RECOMPUTE ? 6 : 3;
    static constexpr bool SW = STAGED && ROWSW;
    static constexpr size_t cube_bytes = (size_t)arrays * EPB * Lay<SW>::ES * sizeof(Real);
    // stage words per field: a tile's chunk of EPB NQ points, or, where chunks
    // do not start on 16-byte boundaries, the window that starts at the chunk's
    // first word rounded down to one and ends on one (the field strides are
    // padded to 32 points, and the point arrays carry slack behind the last)
    static constexpr int VW = 16 / (int)sizeof(Real);
    static constexpr int FE = (EPB * NQ) % VW == 0 ? EPB * NQ : (EPB * NQ + 2 * VW - 2) / VW * VW;
    static constexpr size_t field_bytes = (size_t)FE * sizeof(Real);
    static constexpr size_t bytes =
        (cube_bytes + 15) / 16 * 16 + (STAGED ? (size_t)QpFields<LAW, STORAGE>::n * field_bytes : 0);
};

// ---- mbarrier + bulk-copy staging (Hopper/Blackwell async proxy) ------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Wait for the phase of the given parity; gives up after 2^20 polls or
// `limit` clock cycles (the mesh's wait_limit, 2^32 by default) and returns
// false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit) {
    const uint32_t a = smem_u32(bar);
    const long long t0 = clock64();
    if (limit <= 0) limit = 1ll << 32;
    for (int it = 0;; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (it >= (1 << 20) || clock64() - t0 > limit) return false;
    }
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}
// The bulk copies of a tile's quadrature-point fields into the CTA's stage
// (per field, the tile's chunk of points widened to 16-byte boundaries: it
// starts (e0 NQ) mod (16 / sizeof(Real)) words into the stage field), on the
// CTA's mbarrier, issued by the 32 lanes of one warp (lane f copies fields
// f, f + 32, ...; lane 0 first posts the expected bytes). Called by all lanes
// of that warp after the CTA barrier that ends the stage's previous use; the
// proxy fence orders those generic reads before the copies.
template <int EPB, int LAW, int STORAGE>
__device__ __forceinline__ void stage_issue_warp(const hx::MeshView &m, int tile, Real *stg, uint64_t *bar, int lane) {
    using QF = QpFields<LAW, STORAGE>;
    using SM = ApplySmem<EPB, LAW, STORAGE, true>;
    constexpr int FE = SM::FE;  // stage words per field
    const int e0 = tile * EPB;
    const int cnt = min(EPB, m.n_elem - e0);
    const int64_t c0 = (int64_t)e0 * NQ;
    const int off = FE == EPB * NQ ? 0 : (int)(c0 % SM::VW);  // the chunk's first word in its window
    const uint32_t bytes = (uint32_t)(((off + cnt * NQ) * (int)sizeof(Real) + 15) / 16 * 16);
    static_assert((((FE == EPB * NQ ? 0 : SM::VW - 1) + EPB * NQ) * (int)sizeof(Real) + 15) / 16 * 16 <=
                      FE * (int)sizeof(Real),
                  "the widest window fits its stage field");
    static_assert(2 * SM::VW * (int)sizeof(Real) <= HX_ARRAY_SLACK, "windows stay inside the point arrays");
    if (m.skip_stage_copies) return;  // test hook: the stage never fills and the wait runs out
    if (lane == 0) mbar_expect_tx(bar, QF::n * bytes);
    __syncwarp();
    if (lane < QF::n) {
        const uint64_t pol = policy_evict_first();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
#pragma unroll 1
        for (int f = lane; f < QF::n; f += 32) {
            const Real *src = f < QF::ng ? (const Real *)m.geo + (int64_t)f * m.qs + (c0 - off)
                                         : (const Real *)m.qp + (int64_t)(f - QF::ng) * m.qs + (c0 - off);
            bulk_g2s(stg + f * FE, src, bytes, bar, pol);
        }
    }
}

// Test-gradient integration of the per-point coefficients Q (x, y, z parts in
// X0, X1, X2, overwritten) back to nodal values and the atomic scatter into
// out: Dz^T and Dy^T in place, then Bx^T (Dx^T Qx + .) in place, By^T, Bz^T
// and the scatter from registers. Called after a CTA barrier.
__device__ __forceinline__ void col_backward(const hx::MeshView &m, Real *X0, Real *X1, Real *X2, bool act, bool valid,
                                             int eoff, int a0, int a1, int e, Real *__restrict__ out,
                                             uint64_t pol_keep) {
    Real x[N], y[N], w[N];
    const int o0 = eoff + line_off<0>(a0, a1), o1 = eoff + line_off<1>(a0, a1), o2 = eoff + line_off<2>(a0, a1);
    if (act) {  // in place: z-lines X2 = Dz^T X2, y-lines X1 = Dy^T X1
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ld_line<2>(X2 + c * CCZ + o2, x);
            mv<TD, true>(x, y);
            st_line<2>(X2 + c * CCZ + o2, y);
            ld_line<1>(X1 + c * CCZ + o1, x);
            mv<TD, true>(x, y);
            st_line<1>(X1 + c * CCZ + o1, y);
        }
    }
    __syncthreads();
    if (act) {  // x-lines, in place: X0 = Bx^T (Dx^T X0 + X1 + X2)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ld_line<0>(X0 + c * CCZ + o0, x);
            mv<TD, true>(x, y);
            ld_line<0>(X1 + c * CCZ + o0, w);
#pragma unroll
            for (int k = 0; k < N; ++k) y[k] += w[k];
            ld_line<0>(X2 + c * CCZ + o0, w);
#pragma unroll
            for (int k = 0; k < N; ++k) w[k] += y[k];
            mv<TB, true>(w, y);
            st_line<0>(X0 + c * CCZ + o0, y);
        }
    }
    __syncthreads();
    if (act) {  // y-lines: X1 = By^T X0
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ld_line<1>(X0 + c * CCZ + o1, x);
            mv<TB, true>(x, y);
            st_line<1>(X1 + c * CCZ + o1, y);
        }
    }
    __syncthreads();
    if (valid) {  // z-lines: r = Bz^T X1, scattered from registers
        const int64_t base = elem_base(m, e);
        const bool msk = m.dmask != nullptr;
        Real *eo = m.elem_out ? (Real *)m.elem_out + 3 * ((int64_t)e * NQ + a0 + N * a1) : nullptr;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ld_line<2>(X1 + c * CCZ + o2, x);
            mv<TB, true>(x, y);
#pragma unroll
            for (int k = 0; k < N; ++k) {
                if (eo) {  // ordered assembly: the gather pass sums and masks
                    eo[3 * NN * k + c] = y[k];
                    continue;
                }
                const int64_t d = 3 * node_at(m, base, a0, a1, k) + c;
                if (!(msk && m.dmask[d])) red_add(out + d, y[k], pol_keep);
            }
        }
    }
}

// Backward sweeps after the column-ordered quadrature-point phase: X0 holds
// Qx, X2 holds Qy and rz[c] = Dz^T Qz of each thread's z-line (registers).
// Dy^T in place on X2 and rz into X1, then X0 = Bx^T (Dx^T X0 + X1 + X2)
// in place, X1 = By^T X0 and the scatter of Bz^T X1. Called after a barrier.
template <bool SW, bool WS = false>
__device__ __forceinline__ void col_backward_c(const hx::MeshView &m, Real *X0, Real *X1, Real *X2, Real (*rz)[N],
                                               bool act, bool valid, int eoff, const LineOffs<SW> &o, int a0, int a1,
                                               int e, Real *__restrict__ out, uint64_t pol_keep,
                                               int64_t base_e = -1) {
    constexpr int CZ = Lay<SW>::CZ;
    constexpr bool EO = true;  // even-odd sweeps in the staged apply (see mv)
    Real x[3][N], y[3][N], w[3][N];
    if (act) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int t = 0; t < N; ++t) x[c][t] = X2[eoff + c * CZ + o.y[t]];
        mv3<TD, true, EO>(x, y);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int t = 0; t < N; ++t) {
                X1[eoff + c * CZ + o.z[t]] = rz[c][t];
                X2[eoff + c * CZ + o.y[t]] = y[c][t];
            }
    }
    phase_sync<WS>();
    if (act) {  // x-lines, in place: X0 = Bx^T (Dx^T X0 + X1 + X2)
        Real s1[3][N], s2[3][N];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int t = 0; t < N; ++t) {
                x[c][t] = X0[eoff + c * CZ + o.x + t];
                s1[c][t] = X1[eoff + c * CZ + o.x + t];
                s2[c][t] = X2[eoff + c * CZ + o.x + t];
            }
        mv3<TD, true, EO>(x, y);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int k = 0; k < N; ++k) w[c][k] = y[c][k] + s1[c][k] + s2[c][k];
        mv3<TB, true, EO>(w, y);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int t = 0; t < N; ++t) X0[eoff + c * CZ + o.x + t] = y[c][t];
    }
    phase_sync<WS>();
    if (act) {  // y-lines: X1 = By^T X0
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int t = 0; t < N; ++t) x[c][t] = X0[eoff + c * CZ + o.y[t]];
        mv3<TB, true, EO>(x, y);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int t = 0; t < N; ++t) X1[eoff + c * CZ + o.y[t]] = y[c][t];
    }
    phase_sync<WS>();
    if (valid) {  // z-lines: r = Bz^T X1, scattered from registers
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int t = 0; t < N; ++t) x[c][t] = X1[eoff + c * CZ + o.z[t]];
        mv3<TB, true, EO>(x, y);
        if (m.elem_out) {  // ordered assembly: the gather pass sums and masks
            Real *eo = (Real *)m.elem_out + 3 * ((int64_t)e * NQ + a0 + N * a1);
#pragma unroll
            for (int k = 0; k < N; ++k)
#pragma unroll
                for (int c = 0; c < 3; ++c) eo[3 * NN * k + c] = y[c][k];
            return;
        }
        const int64_t base = base_e >= 0 ? base_e : elem_base(m, e);  // the caller's copy, if it has one
        const bool msk = m.dmask != nullptr;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int64_t d = 3 * node_at(m, base, a0, a1, k);
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (!(msk && m.dmask[d + c])) red_add(out + d + c, y[c][k], pol_keep);
        }
    }
}

// Per-point tangent flux Q from the reference gradient Gr and the point's
// fields r (geometry first unless spatial, then the cache; for the recompute
// strategy Gu is the reference gradient of u_k).
template <int LAW, int STORAGE>
__device__ __forceinline__ void qp_tangent(const hx::MeshView &m, int e, const Real *Gr, const Real *Gu, const Real *r,
                                           Real *Q) {
    if constexpr (STORAGE == HX_SPATIAL_TENSORS) {
        spatial_Q<Real, LAW>(Gr, [&](int f) { return r[f]; }, Q);
    } else {
        Real Ji[9], H[9], dP[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Ji[k] = r[k];
        const Real JxW = r[9];
        State<Real> st;
        if constexpr (STORAGE == HX_RECOMPUTE) {
            push_grad(Gu, Ji, st.Hk);
            state_from_Hk<Real, LAW, (bool)HX_UNIT_F32>(m, e, st);
        } else {
            build_state<Real, LAW, STORAGE>(m, e, [&](int f) { return r[10 + f]; }, st);
        }
        push_grad(Gr, Ji, H);
        tangent_dP<Real, LAW>(st, H, dP);
        pull_flux(dP, Ji, JxW, Q);
    }
}

// Quadrature-point phase of the column-ordered staged apply: thread (a0, a1)
// of an element handles its points (a0, a1, k), k = 0..N-1, whose fields sit
// in the stage at sp[f * FS + NN * k]; Gx, Gy come from X0, X2 at the
// z-line points and Gz from gz (registers); Q_x, Q_y go back to X0, X2 and
// Q_z to gz. Recompute: the reference gradient of u_k from K0, K2, gk.
template <int LAW, int STORAGE, int FS, bool SW>
__device__ __forceinline__ void qp_columns(const hx::MeshView &m, int e, bool valid, const Real *sp, Real *X0,
                                           Real *X2, const Real *K0, const Real *K2, Real (*gz)[N],
                                           const Real (*gk)[N], int eoff, const LineOffs<SW> &lo) {
    constexpr bool RC = STORAGE == HX_RECOMPUTE;
    constexpr int CZ = Lay<SW>::CZ;
    constexpr int NR = QpFields<LAW, STORAGE>::n;
    if constexpr (STORAGE == HX_SPATIAL_TENSORS && PK) {
        // FP32 spatial tensors: the column's points run two at a time in
        // the two lanes of the packed FP32 instructions (points k, k+1;
        // an odd last point alone); the next pair's shared loads are
        // issued before this pair's stores
        if (valid) {
            Real ra[NR], rb[NR], Ga[6], Gb[6];
            auto fetch1 = [&](int k, Real *r, Real *G) {
#pragma unroll
                for (int f = 0; f < NR; ++f) r[f] = sp[f * FS + NN * k];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    G[c] = X0[eoff + lo.z[k] + c * CZ];
                    G[3 + c] = X2[eoff + lo.z[k] + c * CZ];
                }
            };
            fetch1(0, ra, Ga);
            if (N > 1) fetch1(1, rb, Gb);
#pragma unroll
            for (int k = 0; k + 1 < N; k += 2) {
                F2 G2[9], Q2[9];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    G2[c * 3 + 0] = F2(Ga[c], Gb[c]);
                    G2[c * 3 + 1] = F2(Ga[3 + c], Gb[3 + c]);
                    G2[c * 3 + 2] = F2(gz[c][k], gz[c][k + 1]);
                }
                spatial_Q<F2, LAW>(G2, [&](int f) { return F2(ra[f], rb[f]); }, Q2);
                if (k + 2 < N) fetch1(k + 2, ra, Ga);
                if (k + 3 < N) fetch1(k + 3, rb, Gb);
                const int pk = eoff + lo.z[k], pk1 = eoff + lo.z[k + 1];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    X0[pk + c * CZ] = Q2[c * 3 + 0].v.x;
                    X2[pk + c * CZ] = Q2[c * 3 + 1].v.x;
                    X0[pk1 + c * CZ] = Q2[c * 3 + 0].v.y;
                    X2[pk1 + c * CZ] = Q2[c * 3 + 1].v.y;
                    gz[c][k] = Q2[c * 3 + 2].v.x;
                    gz[c][k + 1] = Q2[c * 3 + 2].v.y;
                }
            }
            if constexpr (N % 2 == 1) {  // the last point alone (fetched into ra, Ga)
                constexpr int k = N - 1;
                Real Gr[9], Q[9];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    Gr[c * 3 + 0] = Ga[c];
                    Gr[c * 3 + 1] = Ga[3 + c];
                    Gr[c * 3 + 2] = gz[c][k];
                }
                spatial_Q<Real, LAW>(Gr, [&](int f) { return ra[f]; }, Q);
                const int pk = eoff + lo.z[k];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    X0[pk + c * CZ] = Q[c * 3 + 0];
                    X2[pk + c * CZ] = Q[c * 3 + 1];
                    gz[c][k] = Q[c * 3 + 2];
                }
            }
        }
    } else if (valid) {
        // point k+1's shared loads are issued before point k's stores
        Real r[NR], Gx[3], Gy[3], Ux[3], Uy[3];
        auto fetch = [&](int k) {
#pragma unroll
            for (int f = 0; f < NR; ++f) r[f] = sp[f * FS + NN * k];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Gx[c] = X0[eoff + lo.z[k] + c * CZ];
                Gy[c] = X2[eoff + lo.z[k] + c * CZ];
                if constexpr (RC) {
                    Ux[c] = K0[eoff + lo.z[k] + c * CZ];
                    Uy[c] = K2[eoff + lo.z[k] + c * CZ];
                }
            }
        };
        fetch(0);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            Real Gr[9], Gu[9], Q[9];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Gr[c * 3 + 0] = Gx[c];
                Gr[c * 3 + 1] = Gy[c];
                Gr[c * 3 + 2] = gz[c][k];
                if constexpr (RC) {
                    Gu[c * 3 + 0] = Ux[c];
                    Gu[c * 3 + 1] = Uy[c];
                    Gu[c * 3 + 2] = gk[c][k];
                }
            }
            qp_tangent<LAW, STORAGE>(m, e, Gr, Gu, r, Q);
            if (k + 1 < N) fetch(k + 1);
            const int pk = eoff + lo.z[k];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                X0[pk + c * CZ] = Q[c * 3 + 0];
                X2[pk + c * CZ] = Q[c * 3 + 1];
                gz[c][k] = Q[c * 3 + 2];
            }
        }
    }
}

// One tile (EPB elements, starting at element tile*EPB) of the tangent apply
// on NT threads: forward sum factorization from the x-rows of du (and u_k) that
// each thread holds in cd (ck), the quadrature-point phase, the transposed
// sweeps and the atomic scatter into out. Consecutive calls need no barrier
// between them (see col_forward).
// Quadrature-point phase: flat over the tile's EPB*NQ points (consecutive
// threads take consecutive points). STAGED: the fields were copied into the
// shared stage by bulk copies on `bar` (issued a tile earlier); the copies of
// tile `ntile` (< 0: none) are issued once the stage is consumed. Otherwise
// each thread requests its next point's fields one point ahead. Returns false
// (on every thread) if the staged data never arrived.
template <int EPB, int NT, int LAW, int STORAGE, bool STAGED>
__device__ __forceinline__ bool apply_tile(const hx::MeshView &m, int tile, int ntile, Real *__restrict__ out,
                                           const Real *cd, const Real *ck, unsigned char *smem_raw, Real *stg,
                                           uint64_t *bar, uint32_t &phase, uint64_t pol_keep, uint64_t pol_stream) {
    constexpr bool SW = STAGED && ROWSW;  // row-swizzled cubes, one warp per element
    constexpr int ES = Lay<SW>::ES;
    Real *X0 = (Real *)smem_raw;
    Real *X1 = X0 + EPB * ES;
    Real *X2 = X1 + EPB * ES;
    Real *K0 = X2 + EPB * ES;  // recompute strategy: reference gradient of u_k
    Real *K1 = K0 + EPB * ES;
    Real *K2 = K1 + EPB * ES;
    const int t = threadIdx.x;
    int el, a0, a1;
    bool act;
    thread_map<SW>(t, EPB, el, a0, a1, act);
    const int eoff = (act ? el : 0) * ES;
    constexpr bool RC = STORAGE == HX_RECOMPUTE;
    using QF = QpFields<LAW, STORAGE>;
    constexpr int NR = QF::n;
    const int e0 = tile * EPB;
    const int e = e0 + el;
    const bool valid = act && e < m.n_elem;
    const int nval = min(EPB, m.n_elem - e0) * NQ;  // valid points of this tile
    const int64_t g0 = (int64_t)e0 * NQ;
    auto load_raw = [&](int q, Real *r) {
        const Real *geo = (const Real *)m.geo + g0 + q;
#pragma unroll
        for (int f = 0; f < QF::ng; ++f) r[f] = ld_stream(geo + (int64_t)f * m.qs, pol_stream);
        const Real *qp = (const Real *)m.qp + g0 + q;
#pragma unroll
        for (int f = 0; f < QF::nc; ++f) r[QF::ng + f] = ld_stream(qp + (int64_t)f * m.qs, pol_stream);
    };
    auto point = [&](int q, const Real *r) {
        const int qel = q / NQ;
        const int ql = q - qel * NQ;
        const int pos = qel * CES + (ql % N) + ((ql / N) % N) * CRS + (ql / NN) * CPS;
        Real Gr[9], Gu[9], Q[9];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Gr[c * 3 + 0] = X0[pos + c * CCZ];
            Gr[c * 3 + 1] = X1[pos + c * CCZ];
            Gr[c * 3 + 2] = X2[pos + c * CCZ];
            if constexpr (RC) {
                Gu[c * 3 + 0] = K0[pos + c * CCZ];
                Gu[c * 3 + 1] = K1[pos + c * CCZ];
                Gu[c * 3 + 2] = K2[pos + c * CCZ];
            }
        }
        qp_tangent<LAW, STORAGE>(m, e0 + qel, Gr, Gu, r, Q);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            X0[pos + c * CCZ] = Q[c * 3 + 0];
            X1[pos + c * CCZ] = Q[c * 3 + 1];
            X2[pos + c * CCZ] = Q[c * 3 + 2];
        }
    };
    if constexpr (STAGED) {
        // column order: thread (a0, a1) of element el handles the points
        // (a0, a1, k) of its z-line; the stage holds them at el*NQ + a0 +
        // N*a1 + NN*k (consecutive threads, consecutive words)
        constexpr int CZ = Lay<SW>::CZ;
        const LineOffs<SW> lo = line_offsets<SW>(a0, a1);
        Real gz[3][N], gk[RC ? 3 : 1][N];
        if constexpr (RC) col_forward_c<SW>(ck, K0, K1, K2, gk, act, eoff, lo);
        col_forward_c<SW>(cd, X0, X1, X2, gz, act, eoff, lo);
        const bool ok = mbar_wait(bar, phase, m.wait_limit);
        if (__syncthreads_or(!ok)) {  // also the barrier that completes the forward sweeps
            if (t == 0) {
                atomicOr(m.err + 2, 1);
                mbar_wait(bar, phase, m.wait_limit);  // let a copy still in flight land before the CTA exits
            }
            return false;
        }
        phase ^= 1u;
        using SMS = ApplySmem<EPB, LAW, STORAGE, true>;
        const int soff = SMS::FE == EPB * NQ ? 0 : (int)(((int64_t)tile * EPB * NQ) % SMS::VW);  // chunk in its window
        qp_columns<LAW, STORAGE, SMS::FE, SW>(m, e, valid, stg + soff + el * NQ + a0 + N * a1, X0, X2, K0, K2, gz,
                                              gk, eoff, lo);
        Real rz[3][N];
        mv3<TD, true, true>(gz, rz);
        __syncthreads();
        if (t < 32 && ntile >= 0) stage_issue_warp<EPB, LAW, STORAGE>(m, ntile, stg, bar, t);
        col_backward_c<SW>(m, X0, X1, X2, rz, act, valid, eoff, lo, a0, a1, e, out, pol_keep);
        return true;
    } else {
        Real rc[NR], rn[NR];
        if (t < nval) load_raw(t, rc);
        if constexpr (RC) col_forward(ck, K0, K1, K2, act, eoff, a0, a1);
        col_forward(cd, X0, X1, X2, act, eoff, a0, a1);
        __syncthreads();
#pragma unroll 1
        for (int q = t; q < nval; q += NT) {
            if (q + NT < nval) load_raw(q + NT, rn);
            point(q, rc);
#pragma unroll
            for (int f = 0; f < NR; ++f) rc[f] = rn[f];
        }
        __syncthreads();
    }
    col_backward(m, X0, X1, X2, act, valid, eoff, a0, a1, e, out, pol_keep);
    return true;
}

// ---------------------------------------------------------------------------
// Warp-decoupled staged apply (variants 2 and 5, FP32 up to n = 5): every warp
// owns a group of WEPW whole elements (one row-swizzled element at n = 5;
// 32 / n^2 column-layout elements below) with its own stage and mbarrier, so
// no phase needs more than a warp barrier and the warps of a CTA drift
// freely. A group's chunk of a field (WEPW * NQ words) need not start on a
// 16-byte boundary, so the warp copies the window of WWIN words that starts
// at the chunk's first word rounded down to a multiple of 4 (the neighbours'
// edge words come along unused; they lie in sectors the neighbouring group
// reads anyway) and reads from word (first word mod 4) of the window.
// ---------------------------------------------------------------------------
constexpr int WEPW = ROWSW ? 1 : (NN <= 32 ? 32 / NN : 0);  // elements per warp (0: not built)
constexpr int WCH = WEPW * NQ;                              // words of a group's chunk of one field
constexpr int WWIN = WCH % 4 == 0 ? WCH : (WCH + 6) / 4 * 4;  // window words: covers a shift of up to 3
constexpr bool WD_OK = sizeof(Real) == 4 && WEPW > 0;
// A window reaches at most WWIN - NQ words past the last element's points;
// the point arrays carry HX_ARRAY_SLACK bytes after their last field.
static_assert(!WD_OK || (WWIN - NQ) * 4 <= HX_ARRAY_SLACK, "stage windows would leave the point arrays");

// The bulk copies of group g's point fields into the warp's stage (one
// WWIN-word window per field), on the warp's mbarrier, issued by the whole
// warp (lane f copies fields f, f + 32, ...; lane 0 first posts the expected
// bytes). Called by all 32 lanes after the warp barrier that ends the stage's
// previous use.
template <int LAW, int STORAGE>
__device__ __forceinline__ void stage_issue_group(const hx::MeshView &m, int g, Real *stg, uint64_t *bar, int lane) {
    using QF = QpFields<LAW, STORAGE>;
    static_assert(LAW >= 0 && WD_OK, "the window layout is that of FP32 groups of whole elements in one warp");
    if (m.skip_stage_copies) return;  // test hook: the stage never fills and the wait runs out
    const int64_t c0 = (int64_t)g * WCH;
    const int64_t w0 = c0 - (c0 & 3);  // first word of the window: a multiple of 4
    if (lane == 0) mbar_expect_tx(bar, QF::n * WWIN * 4);
    __syncwarp();
    if (lane < QF::n) {
        const uint64_t pol = policy_evict_first();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
#pragma unroll 1
        for (int f = lane; f < QF::n; f += 32) {
            const Real *src = f < QF::ng ? (const Real *)m.geo + (int64_t)f * m.qs + w0
                                         : (const Real *)m.qp + (int64_t)(f - QF::ng) * m.qs + w0;
            bulk_g2s(stg + f * WWIN, src, WWIN * 4, bar, pol);
        }
    }
}

// Shared-memory bytes of a CTA of W warps: the cubes of its W * WEPW elements,
// then the W stages.
template <int W, int LAW, int STORAGE>
__host__ __device__ constexpr size_t wd_cubes_bytes() {
    return ((size_t)3 * W * WEPW * Lay<ROWSW>::ES * sizeof(Real) + 15) / 16 * 16;
}
template <int W, int LAW, int STORAGE>
__host__ __device__ constexpr size_t wd_smem_bytes() {
    return wd_cubes_bytes<W, LAW, STORAGE>() + (size_t)W * QpFields<LAW, STORAGE>::n * WWIN * sizeof(Real);
}

// out += K(u_k) du, one group of WEPW elements per warp with its own stage
// (caching strategies). Warp w of a CTA takes group tile*W + w of each of the
// CTA's tiles (elements g*WEPW .. g*WEPW + WEPW - 1); the warp issues the
// copies of its next group as soon as it has consumed its stage.
template <int W, int LAW, int STORAGE>
__global__ void __launch_bounds__(W * 32) k_apply_wd(const hx::MeshView m, const Real *__restrict__ du,
                                                     Real *__restrict__ out, int ntiles) {
    static_assert(WD_OK && STORAGE != HX_RECOMPUTE, "FP32 groups of whole elements per warp, caching strategies");
    constexpr bool SW = ROWSW;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[W];
    using QF = QpFields<LAW, STORAGE>;
    constexpr int ES = Lay<SW>::ES;
    const int t = threadIdx.x;
    const int wid = t >> 5, lane = t & 31;
    const int sub = lane / NN;  // element of the group
    const bool act = sub < WEPW;
    const int a = act ? lane - sub * NN : 0;
    const int a0 = a % N, a1 = a / N;
    const int eoff = (wid * WEPW + (act ? sub : 0)) * ES;
    Real *X0 = (Real *)smem_raw;
    Real *X1 = X0 + W * WEPW * ES;
    Real *X2 = X1 + W * WEPW * ES;
    Real *stg = (Real *)(smem_raw + wd_cubes_bytes<W, LAW, STORAGE>()) + wid * (QF::n * WWIN);
    uint64_t *bar = &bars[wid];
    const uint64_t pol_keep = policy_evict_last();
    const LineOffs<SW> lo = line_offsets<SW>(a0, a1);
    uint32_t phase = 0;
    if (lane == 0) mbar_init(bar, 1);
    __syncwarp();
    const int stride = gridDim.x * W;  // groups
    int g = blockIdx.x * W + wid;
    int e = g * WEPW + sub;
    if ((int)blockIdx.x < ntiles && g * WEPW < m.n_elem) stage_issue_group<LAW, STORAGE>(m, g, stg, bar, lane);
    Real row[3 * N];
    int64_t base = elem_base(m, e);  // 0 past the end
    if (act) load_row(m, e, base, a0, a1, du, true, row);  // zeros past the end
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, g += stride, e += stride * WEPW) {
        if (g * WEPW >= m.n_elem) break;  // warp-uniform; later tiles lie further out
        const bool valid = act && e < m.n_elem;
        const int gn = g + stride;
        const int en = e + stride * WEPW;
        Real cd[3 * N];
#pragma unroll
        for (int i = 0; i < 3 * N; ++i) cd[i] = row[i];
        const int64_t base_n = elem_base(m, en);
        if (act) load_row(m, en, base_n, a0, a1, du, true, row);
        Real gz[3][N], gk[1][N];
        col_forward_c<SW, true>(cd, X0, X1, X2, gz, act, eoff, lo);
        const bool ok = mbar_wait(bar, phase, m.wait_limit);
        if (__any_sync(0xffffffffu, !ok)) {
            if (lane == 0) {
                atomicOr(m.err + 2, 1);
                mbar_wait(bar, phase, m.wait_limit);  // let a copy still in flight land before the warp exits
            }
            return;
        }
        __syncwarp();  // completes the forward sweeps
        phase ^= 1u;
        qp_columns<LAW, STORAGE, WWIN, SW>(m, e, valid, stg + (int)(((int64_t)g * WCH) & 3) + sub * NQ + a0 + N * a1,
                                           X0, X2, nullptr, nullptr, gz, gk, eoff, lo);
        Real rz[3][N];
        mv3<TD, true, true>(gz, rz);
        __syncwarp();  // the stage is consumed
        if (gn * WEPW < m.n_elem) stage_issue_group<LAW, STORAGE>(m, gn, stg, bar, lane);
        col_backward_c<SW, true>(m, X0, X1, X2, rz, act, valid, eoff, lo, a0, a1, e, out, pol_keep, base);
        base = base_n;
    }
}

// One tile of the residual R(u) (same structure as apply_tile): the state is
// rebuilt at every point from the forward gradient of u (Hk = Grad u), then
// P = (I + Hk) S and Q = JxW P J0^-T. Geometry is read with a one-point-ahead
// register prefetch.
template <int EPB, int NT, int LAW>
__device__ __forceinline__ void residual_tile(const hx::MeshView &m, int tile, Real *__restrict__ out,
                                              const Real *cu, unsigned char *smem_raw, uint64_t pol_keep,
                                              uint64_t pol_stream) {
    Real *X0 = (Real *)smem_raw;
    Real *X1 = X0 + EPB * CES;
    Real *X2 = X1 + EPB * CES;
    const int t = threadIdx.x;
    const int el = t / NN;
    const int a = t - el * NN;
    const int a0 = a % N, a1 = a / N;
    const bool act = el < EPB;
    const int eoff = (act ? el : 0) * CES;
    const int e0 = tile * EPB;
    const int e = e0 + el;
    const bool valid = act && e < m.n_elem;
    const int nval = min(EPB, m.n_elem - e0) * NQ;
    const int64_t g0 = (int64_t)e0 * NQ;
    Real rc[10], rn[10];
    auto load_geo_raw = [&](int q, Real *r) {
        const Real *geo = (const Real *)m.geo + g0 + q;
#pragma unroll
        for (int f = 0; f < 10; ++f) r[f] = ld_stream(geo + (int64_t)f * m.qs, pol_stream);
    };
    if (t < nval) load_geo_raw(t, rc);
    col_forward(cu, X0, X1, X2, act, eoff, a0, a1);
    __syncthreads();
#pragma unroll 1
    for (int q = t; q < nval; q += NT) {
        if (q + NT < nval) load_geo_raw(q + NT, rn);
        const int qel = q / NQ;
        const int ql = q - qel * NQ;
        const int pos = qel * CES + (ql % N) + ((ql / N) % N) * CRS + (ql / NN) * CPS;
        Real Ji[9], Gr[9], P[9], Q[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Ji[k] = rc[k];
        const Real JxW = rc[9];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Gr[c * 3 + 0] = X0[pos + c * CCZ];
            Gr[c * 3 + 1] = X1[pos + c * CCZ];
            Gr[c * 3 + 2] = X2[pos + c * CCZ];
        }
        State<Real> st;
        push_grad(Gr, Ji, st.Hk);
        state_from_Hk<Real, LAW, (bool)HX_UNIT_F32>(m, e0 + qel, st);
        flag_state(m, (double)st.Jm1);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                Real s = st.S[SI(c, d)];
#pragma unroll
                for (int k = 0; k < 3; ++k) s = fma(st.Hk[c * 3 + k], st.S[SI(k, d)], s);
                P[c * 3 + d] = s;
            }
        pull_flux(P, Ji, JxW, Q);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            X0[pos + c * CCZ] = Q[c * 3 + 0];
            X1[pos + c * CCZ] = Q[c * 3 + 1];
            X2[pos + c * CCZ] = Q[c * 3 + 2];
        }
#pragma unroll
        for (int f = 0; f < 10; ++f) rc[f] = rn[f];
    }
    __syncthreads();
    col_backward(m, X0, X1, X2, act, valid, eoff, a0, a1, e, out, pol_keep);
}

// r += R(u) over all elements (r zeroed by the caller); persistent like
// k_apply, with the rows of u (Dirichlet values included) one tile ahead.
template <int EPB, int LAW>
__global__ void __launch_bounds__(col_threads(EPB)) k_residual_col(const hx::MeshView m, const Real *__restrict__ u,
                                                                   Real *__restrict__ r, int ntiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int t = threadIdx.x;
    const int el = t / NN;
    const int a = t - el * NN;
    const int a0 = a % N, a1 = a / N;
    const bool act = el < EPB;
    const uint64_t pol_keep = policy_evict_last();
    const uint64_t pol_stream = policy_evict_first();
    Real row[3 * N];  // R needs only Grad u: rows relative to the element's first node (shift_row)
    if (act && (int)blockIdx.x < ntiles) {
        const int e1 = blockIdx.x * EPB + el;
        const int64_t base = elem_base(m, e1);
        load_row(m, e1, base, a0, a1, u, false, row);
        shift_row(m, e1, base, u, row);
    }
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int ntile = tile + gridDim.x;
        Real cu[3 * N];
#pragma unroll
        for (int i = 0; i < 3 * N; ++i) cu[i] = row[i];
        if (act && ntile < ntiles) {
            const int e1 = ntile * EPB + el;
            const int64_t base = elem_base(m, e1);
            load_row(m, e1, base, a0, a1, u, false, row);
            shift_row(m, e1, base, u, row);
        }
        // no barrier: the previous tile's last phase reads X1 only, the first
        // phase of this one writes X0 only
        residual_tile<EPB, col_threads(EPB), LAW>(m, tile, r, cu, smem_raw, pol_keep, pol_stream);
    }
}

// out += K(u_k) du over all elements (out zeroed by the caller). Persistent:
// CTAs walk tiles of EPB elements with stride gridDim.x. Each thread loads
// its element x-row of du (and u_k) straight into registers, one tile ahead.
// STAGED: the tile's quadrature-point fields arrive in shared memory by bulk
// copies issued one tile ahead (a single stage, refilled after each
// quadrature-point phase); a copy that never completes sets the device
// timeout flag and ends the CTA.
template <int EPB, int LAW, int STORAGE, bool STAGED>
__global__ void __launch_bounds__(apply_threads<STAGED && ROWSW>(EPB)) k_apply(const hx::MeshView m,
                                                                               const Real *__restrict__ du,
                                                                               Real *__restrict__ out, int ntiles) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    const int t = threadIdx.x;
    int el, a0, a1;
    bool act;
    thread_map<STAGED && ROWSW>(t, EPB, el, a0, a1, act);
    const uint64_t pol_keep = policy_evict_last();
    const uint64_t pol_stream = policy_evict_first();
    constexpr bool RC = STORAGE == HX_RECOMPUTE;
    using SM = ApplySmem<EPB, LAW, STORAGE, STAGED>;
    Real *stg = (Real *)(smem_raw + (SM::cube_bytes + 15) / 16 * 16);
    uint32_t phase = 0;
    if constexpr (STAGED) {
        if (t == 0) mbar_init(&bar, 1);
        __syncthreads();
        if (t < 32 && (int)blockIdx.x < ntiles) stage_issue_warp<EPB, LAW, STORAGE>(m, blockIdx.x, stg, &bar, t);
    }
    Real rowd[3 * N], rowk[RC ? 3 * N : 1];
    if (act && (int)blockIdx.x < ntiles) {
        const int e1 = blockIdx.x * EPB + el;
        const int64_t b1 = elem_base(m, e1);
        load_row(m, e1, b1, a0, a1, du, true, rowd);
        if constexpr (RC) {  // only Grad u_k is needed (shift_row)
            load_row(m, e1, b1, a0, a1, (const Real *)m.uk, false, rowk);
            shift_row(m, e1, b1, (const Real *)m.uk, rowk);
        }
    }
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int ntile = tile + gridDim.x;
        if (!STAGED && m.l2pf) prefetch_tile<EPB, STORAGE>(m, ntile);
        // this tile's rows; the next tile's rows are requested now
        Real cd[3 * N], ck[RC ? 3 * N : 1];
#pragma unroll
        for (int i = 0; i < 3 * N; ++i) cd[i] = rowd[i];
        if constexpr (RC) {
#pragma unroll
            for (int i = 0; i < 3 * N; ++i) ck[i] = rowk[i];
        }
        if (act && ntile < ntiles) {
            const int e1 = ntile * EPB + el;
            const int64_t b1 = elem_base(m, e1);
            load_row(m, e1, b1, a0, a1, du, true, rowd);
            if constexpr (RC) {
                load_row(m, e1, b1, a0, a1, (const Real *)m.uk, false, rowk);
                shift_row(m, e1, b1, (const Real *)m.uk, rowk);
            }
        }
        // no barrier: the previous tile's last phase reads X1 only, the first
        // phase of this one writes X0 (and K0) only
        if (!apply_tile<EPB, apply_threads<STAGED && ROWSW>(EPB), LAW, STORAGE, STAGED>(m, tile, ntile < ntiles ? ntile : -1, out, cd,
                                                                    ck, smem_raw, stg, &bar, phase, pol_keep,
                                                                    pol_stream))
            return;
    }
}

// One work item of a batch (one tile of one mesh) on NT threads: the rows are
// loaded at the start of the item (no prefetch across items, which may belong
// to meshes of other degrees).
template <int EPB, int NT, int LAW, int STORAGE>
__device__ __forceinline__ void batch_tile(const hx::MeshView &m, int tile, const Real *__restrict__ du,
                                           Real *__restrict__ out, unsigned char *smem_raw) {
    const int t = threadIdx.x;
    const int el = t / NN;
    const int a = t - el * NN;
    const int a0 = a % N, a1 = a / N;
    constexpr bool RC = STORAGE == HX_RECOMPUTE;
    Real cd[3 * N], ck[RC ? 3 * N : 1];
    if (el < EPB) {
        const int e1 = tile * EPB + el;
        const int64_t b1 = elem_base(m, e1);
        load_row(m, e1, b1, a0, a1, du, true, cd);
        if constexpr (RC) {  // only Grad u_k is needed (shift_row)
            load_row(m, e1, b1, a0, a1, (const Real *)m.uk, false, ck);
            shift_row(m, e1, b1, (const Real *)m.uk, ck);
        }
    }
    uint32_t phase = 0;
    apply_tile<EPB, NT, LAW, STORAGE, false>(m, tile, -1, out, cd, ck, smem_raw, nullptr, nullptr, phase,
                                             policy_evict_last(), policy_evict_first());
}

// The same with the quadrature-point fields staged by bulk copies (caching
// strategies): thread 0 issues the item's copies on `bar` when the item starts
// (the caller's CTA barrier has retired the previous item's stage), so they
// overlap the row loads and the forward sweeps; `phase` is the parity of the
// wait. Returns false (on every thread) if the copies never arrived.
template <int EPB, int NT, int LAW, int STORAGE>
__device__ __forceinline__ bool batch_tile_staged(const hx::MeshView &m, int tile, const Real *__restrict__ du,
                                                  Real *__restrict__ out, unsigned char *smem_raw, uint64_t *bar,
                                                  uint32_t phase) {
    static_assert(STORAGE != HX_RECOMPUTE, "the staged tile runs the caching strategies");
    using SM = ApplySmem<EPB, LAW, STORAGE, true>;
    Real *stg = (Real *)(smem_raw + (SM::cube_bytes + 15) / 16 * 16);
    const int t = threadIdx.x;
    if (t < 32) stage_issue_warp<EPB, LAW, STORAGE>(m, tile, stg, bar, t);
    int el, a0, a1;
    bool act;
    thread_map<ROWSW>(t, EPB, el, a0, a1, act);
    Real cd[3 * N], ck[1];
    if (act) {
        const int e1 = tile * EPB + el;
        load_row(m, e1, elem_base(m, e1), a0, a1, du, true, cd);
    }
    return apply_tile<EPB, NT, LAW, STORAGE, true>(m, tile, -1, out, cd, ck, smem_raw, stg, bar, phase,
                                                   policy_evict_last(), policy_evict_first());
}

// qp cache at state u: interpolation and state in FP64, stored as Real
template <int EPB, int LAW, int STORAGE>
__global__ void __launch_bounds__(threads_for(EPB)) k_precompute(const hx::MeshView m, const double *__restrict__ u, Real *__restrict__ qp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *U = (double *)smem_raw;
    double *W = U + 3 * EPB * SZ;
    double *G = W + 3 * EPB * SZ;
    const int e0 = blockIdx.x * EPB;
    constexpr int nc = 3 * EPB;
    gather(m, e0, EPB, u, U, false);
    __syncthreads();
    forward_grad(U, W, G, nc);
    const double *geo = m.geo64;  // FP64 geometry always
    for (int it = threadIdx.x; it < EPB * NQ; it += blockDim.x) {
        const int el = it / NQ;
        const int q = it - el * NQ;
        const int e = e0 + el;
        if (e >= m.n_elem) continue;
        const int ci = cidx(q % N, (q / N) % N, q / NN);
        const int64_t g = (int64_t)e * NQ + q;
        double Ji[9], Gr[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Ji[k] = geo[(int64_t)k * m.qs + g];
#pragma unroll
        for (int k = 0; k < 9; ++k) Gr[k] = G[(el * 9 + k) * SZ + ci];
        State<double> st;
        push_grad(Gr, Ji, st.Hk);
        state_from_Hk<double, LAW, false>(m, e, st);
        flag_state(m, st.Jm1);
        if constexpr (STORAGE == HX_SPATIAL_TENSORS) {
            double f[hx::qp_fields(LAW, STORAGE)];
            spatial_fields<LAW>(st, Ji, geo[(int64_t)9 * m.qs + g], m, f);
#pragma unroll
            for (int k = 0; k < hx::qp_fields(LAW, STORAGE); ++k) qp[(int64_t)k * m.qs + g] = (Real)f[k];
        } else if constexpr (STORAGE != HX_RECOMPUTE) {
            store_state<Real, LAW, STORAGE>(qp, m.qs, g, st);
        }
    }
}

// Diagonal: per qp the 3 blocks A_c[d][f] = d(dP_cd)/d(H_cf) pulled back to
// reference coordinates, M_c = JxW J0^-1 A_c J0^-T (symmetric), then
// diag_c(a) = sum_q grad_xi N_a^T M_c grad_xi N_a by sum factorization with
// products of the 1D tables.
template <int LAW, int STORAGE>
__global__ void __launch_bounds__(threads_for(2)) k_diagonal(const hx::MeshView m, Real *__restrict__ diag) {
    constexpr int EPB = 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *U = (Real *)smem_raw;
    Real *W = U + 3 * SZ;
    Real *Gk = W + 3 * SZ;
    Real *Mc = Gk + 9 * SZ;   // 18 cubes: (c*6 + pair)
    Real *T1 = Mc + 18 * SZ;  // 18 cubes
    __shared__ Real tabs[3][NN];  // BB, BG, GG  [q][a]
    const int e0 = blockIdx.x;
    for (int i = threadIdx.x; i < NN; i += blockDim.x) {
        const Real b = tab<TB>(i), gd = tab<TG>(i);
        tabs[0][i] = b * b;
        tabs[1][i] = b * gd;
        tabs[2][i] = gd * gd;
    }
    if constexpr (STORAGE == HX_RECOMPUTE) {
        gather(m, e0, EPB, (const Real *)m.uk, U, false);
        __syncthreads();
        forward_grad(U, W, Gk, 3);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NQ; q += blockDim.x) {
        const int e = e0;
        const int ci = cidx(q % N, (q / N) % N, q / NN);
        const int64_t g = (int64_t)e * NQ + q;
        if constexpr (STORAGE == HX_SPATIAL_TENSORS) {
            // M_c[e1][e2] = dQ_{c e1} / dG_{c e2}: Q for G = e_c (x) e_e2
            Real fl[hx::qp_fields(LAW, STORAGE)];
            const Real *qpd = (const Real *)m.qp;
#pragma unroll
            for (int k = 0; k < hx::qp_fields(LAW, STORAGE); ++k) fl[k] = __ldcs(qpd + (int64_t)k * m.qs + g);
#pragma unroll 1
            for (int c = 0; c < 3; ++c) {
#pragma unroll 1
                for (int e2 = 0; e2 < 3; ++e2) {
                    Real Gu[9], Q[9];
#pragma unroll
                    for (int k = 0; k < 9; ++k) Gu[k] = Real(0);
                    Gu[c * 3 + e2] = Real(1);
                    spatial_Q<Real, LAW>(Gu, [&](int f) { return fl[f]; }, Q);
#pragma unroll
                    for (int e1 = 0; e1 < 3; ++e1)
                        if (e1 <= e2) Mc[(c * 6 + SI(e1, e2)) * SZ + ci] = (e1 == e2) ? Q[c * 3 + e1] : Real(2) * Q[c * 3 + e1];
                }
            }
            continue;
        }
        Real Ji[9], JxW;
        load_geo(m, g, Ji, JxW);
        State<Real> st;
        if constexpr (STORAGE == HX_RECOMPUTE) {
            Real Gu[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) Gu[k] = Gk[k * SZ + ci];
            push_grad(Gu, Ji, st.Hk);
            state_from_Hk<Real, LAW, (bool)HX_UNIT_F32>(m, e, st);
        } else {
            load_state<Real, LAW, STORAGE>(m, e, g, st);
        }
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            Real A[9];  // A[d*3+f] = dP_cd for H = e_c (x) e_f
#pragma unroll 1
            for (int f = 0; f < 3; ++f) {
                Real H[9], dP[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) H[k] = Real(0);
                H[c * 3 + f] = Real(1);
                tangent_dP<Real, LAW>(st, H, dP);
#pragma unroll
                for (int d = 0; d < 3; ++d) A[d * 3 + f] = dP[c * 3 + d];
            }
            // M = JxW Ji A Ji^T
            Real T9[9];
#pragma unroll
            for (int e1 = 0; e1 < 3; ++e1)
#pragma unroll
                for (int f = 0; f < 3; ++f) T9[e1 * 3 + f] = fma(Ji[e1 * 3 + 0], A[0 * 3 + f], fma(Ji[e1 * 3 + 1], A[1 * 3 + f], Ji[e1 * 3 + 2] * A[2 * 3 + f]));
#pragma unroll
            for (int e1 = 0; e1 < 3; ++e1)
#pragma unroll
                for (int e2 = e1; e2 < 3; ++e2) {
                    const Real v = JxW * fma(T9[e1 * 3 + 0], Ji[e2 * 3 + 0], fma(T9[e1 * 3 + 1], Ji[e2 * 3 + 1], T9[e1 * 3 + 2] * Ji[e2 * 3 + 2]));
                    Mc[(c * 6 + SI(e1, e2)) * SZ + ci] = (e1 == e2) ? v : Real(2) * v;
                }
        }
    }
    __syncthreads();
    // pair (e1,e2) by sym index: 0 (0,0) 1 (1,1) 2 (2,2) 3 (0,1) 4 (0,2) 5 (1,2);
    // for direction d the 1D table is BB, BG or GG by how many of e1, e2 equal d
    auto tsel = [](int pair, int d) {
        const int e1 = pair < 3 ? pair : (pair == 5 ? 1 : 0);
        const int e2 = pair < 3 ? pair : (pair == 3 ? 1 : 2);
        return (e1 == d) + (e2 == d);
    };
    // x then y contraction (q -> a) per cube
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        const Real *in = pass == 0 ? Mc : T1;
        Real *out = pass == 0 ? T1 : Mc;
        for (int l = threadIdx.x; l < 18 * NN; l += blockDim.x) {
            const int cube = l / NN;
            const int r = l - cube * NN;
            const int a = r % N, b = r / N;
            const int off = pass == 0 ? R * (a + N * b) : a + R * N * b;
            const int str = pass == 0 ? 1 : R;
            const Real *tb = tabs[tsel(cube % 6, pass)];
            Real x[N];
#pragma unroll
            for (int t = 0; t < N; ++t) x[t] = in[cube * SZ + off + t * str];
#pragma unroll
            for (int o = 0; o < N; ++o) {
                Real s = Real(0);
#pragma unroll
                for (int t = 0; t < N; ++t) s = fma(tb[t * N + o], x[t], s);
                out[cube * SZ + off + o * str] = s;
            }
        }
        __syncthreads();
    }
    // z contraction summed over the six pairs -> U cube c
    for (int l = threadIdx.x; l < 3 * NN; l += blockDim.x) {
        const int c = l / NN;
        const int r = l - c * NN;
        const int off = (r % N) + R * (r / N);
        Real acc[N];
#pragma unroll
        for (int o = 0; o < N; ++o) acc[o] = Real(0);
#pragma unroll 1
        for (int pair = 0; pair < 6; ++pair) {
            const Real *tb = tabs[tsel(pair, 2)];
            const Real *in = Mc + (c * 6 + pair) * SZ + off;
            Real x[N];
#pragma unroll
            for (int t = 0; t < N; ++t) x[t] = in[t * R * N];
#pragma unroll
            for (int o = 0; o < N; ++o)
#pragma unroll
                for (int t = 0; t < N; ++t) acc[o] = fma(tb[t * N + o], x[t], acc[o]);
        }
#pragma unroll
        for (int o = 0; o < N; ++o) U[c * SZ + off + o * R * N] = acc[o];
    }
    __syncthreads();
    scatter_add(m, e0, EPB, U, diag, true);
}

// ---------------------------------------------------------------------------
// Pointwise law evaluation for the forward-stability study (Sec. 7.1): S,
// P = F S and dP = H S + F D_uS[H] at Grad u = G in this unit's precision.
// FORM 0: the stable forms with J^-2/3 = exp(-2/3 ln_{+1}(J-1)); FORM 1: the
// stable forms with Alg. 2 for J^-2/3; FORM 2: the standard forms, from
// F = I + G, C = F^T F, C^-1 = C^{-1} (adjugate), J = det F, ln J, J^-2/3 by
// pow, E = (C - I)/2 (Sec. 3 and App. A as printed, before the Sec. 4
// rewrites).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T det3(const T *A) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
}
template <typename T>
__device__ __forceinline__ void inv3(const T *A, T *Ai) {
    const T id = T(1) / det3(A);
    Ai[0] = (A[4] * A[8] - A[5] * A[7]) * id;
    Ai[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    Ai[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    Ai[3] = (A[5] * A[6] - A[3] * A[8]) * id;
    Ai[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    Ai[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    Ai[6] = (A[3] * A[7] - A[4] * A[6]) * id;
    Ai[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    Ai[8] = (A[0] * A[4] - A[1] * A[3]) * id;
}
template <typename T>
__device__ __forceinline__ void mm3(const T *A, const T *B, T *C, bool ta = false) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T s = T(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) s += (ta ? A[k * 3 + i] : A[i * 3 + k]) * B[k * 3 + j];
            C[i * 3 + j] = s;
        }
}

template <typename T, int LAW>
__device__ void standard_eval(const hx::MeshView &m, int e, const T *G, const T *H, T *S9, T *P, T *dP) {
    const Mat<T> mp = mat_of<T>(m);
    T F[9], C[9], Ci[9], Fi[9], FtH[9], dC[9], X1[9], dCi[9], dS[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = G[k] + ((k % 4) == 0 ? T(1) : T(0));
    mm3(F, F, C, true);
    inv3(C, Ci);
    inv3(F, Fi);
    const T J = det3(F);
    const T lnJ = log(J);
    const T I1 = C[0] + C[4] + C[8];
    mm3(F, H, FtH, true);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) dC[i * 3 + j] = FtH[i * 3 + j] + FtH[j * 3 + i];
    mm3(Ci, dC, X1);
    mm3(X1, Ci, dCi);
#pragma unroll
    for (int k = 0; k < 9; ++k) dCi[k] = -dCi[k];
    T A[9];
    mm3(Fi, H, A);
    const T t = A[0] + A[4] + A[8];  // (1/J) D_u J
    if constexpr (LAW == HX_CNH) {
        const T a = mp.mu - T(2) * mp.lambda * lnJ;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            S9[k] = -a * Ci[k] + ((k % 4) == 0 ? mp.mu : T(0));
            dS[k] = -a * dCi[k] + T(2) * mp.lambda * t * Ci[k];
        }
    } else {
        const T j23 = pow(J, T(-2.0 / 3.0));
        const T c1 = T(0.5) * mp.kappa * (J * J - T(1)) - mp.mu / T(3) * j23 * I1;
        const T c2 = T(2) * mp.mu / T(9) * j23 * I1 + mp.kappa * J * J;
        const T dI1 = T(2) * (FtH[0] + FtH[4] + FtH[8]);
        const T cC = c2 * t - mp.mu / T(3) * j23 * dI1;
        const T cI = T(-2) * mp.mu / T(3) * j23 * t;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            S9[k] = c1 * Ci[k] + ((k % 4) == 0 ? mp.mu * j23 : T(0));
            dS[k] = c1 * dCi[k] + cC * Ci[k] + ((k % 4) == 0 ? cI : T(0));
        }
        if constexpr (LAW == HX_FIBER) {
            State<T> fs;
            load_fibH(m, e, fs);
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const T *Hs = f ? fs.H6 : fs.H4;
                T Hf[9];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) Hf[i * 3 + j] = Hs[SI(i, j)];
                T HC = T(0), HdC = T(0), Is = T(0);
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    HC += Hf[k] * C[k];
                    HdC += Hf[k] * dC[k];
                }
                T M1[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) M1[d] = (T)m.fibM[(int64_t)(3 * f + d) * m.n_elem + e];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) Is += M1[i] * C[i * 3 + j] * M1[j];
                if (Is > T(1)) {
                    const T E = HC - T(1);
                    const T c3 = T(2) * mp.k1 * exp(mp.k2 * E * E);
                    const T cd = c3 * (T(2) * mp.k2 * E * E + T(1)) * HdC;
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        S9[k] += c3 * E * Hf[k];
                        dS[k] += cd * Hf[k];
                    }
                }
            }
        }
    }
    T HS[9], FdS[9];
    mm3(F, S9, P);
    mm3(H, S9, HS);
    mm3(F, dS, FdS);
#pragma unroll
    for (int k = 0; k < 9; ++k) dP[k] = HS[k] + FdS[k];
}

template <int LAW, int FORM>
__global__ void __launch_bounds__(128) k_material_eval(const hx::MeshView m, int e, int64_t n, const double *__restrict__ G,
                                                       const double *__restrict__ H, double *__restrict__ S,
                                                       double *__restrict__ P, double *__restrict__ dP) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        Real g[9], h[9], s9[9], p9[9], d9[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            g[k] = (Real)G[i * 9 + k];
            h[k] = (Real)H[i * 9 + k];
        }
        if constexpr (FORM == 2) {
            standard_eval<Real, LAW>(m, e, g, h, s9, p9, d9);
        } else {
            State<Real> st;
#pragma unroll
            for (int k = 0; k < 9; ++k) st.Hk[k] = g[k];
            state_from_Hk<Real, LAW, FORM == 1>(m, e, st);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    s9[a * 3 + b] = st.S[SI(a, b)];
                    Real v = st.S[SI(a, b)];
#pragma unroll
                    for (int k = 0; k < 3; ++k) v = fma(st.Hk[a * 3 + k], st.S[SI(k, b)], v);
                    p9[a * 3 + b] = v;
                }
            tangent_dP<Real, LAW>(st, h, d9);
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            S[i * 9 + k] = (double)s9[k];
            P[i * 9 + k] = (double)p9[k];
            dP[i * 9 + k] = (double)d9[k];
        }
    }
}

// External load vector of a constant body force b (Sec. 2, the (v, B) term
// of the residual): f_i += sum_q JxW_q N_i(x_q) b, by the transposed value
// sweeps Bz^T, By^T, Bx^T of JxW b and a scatter (constrained rows skipped).
// FP64 throughout (the geometry's FP64 copy).
template <int EPB>
__global__ void __launch_bounds__(threads_for(EPB)) k_body_force(const hx::MeshView m, double b0, double b1, double b2,
                                                                double *__restrict__ f) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *U = (Real *)smem_raw;
    Real *W = U + 3 * EPB * SZ;
    const int e0 = blockIdx.x * EPB;
    for (int it = threadIdx.x; it < EPB * NQ; it += blockDim.x) {
        const int el = it / NQ;
        const int q = it - el * NQ;
        const int e = e0 + el;
        const int ci = cidx(q % N, (q / N) % N, q / NN);
        const double jxw = e < m.n_elem ? m.geo64[(int64_t)9 * m.qs + (int64_t)e * NQ + q] : 0.0;
        W[(el * 3 + 0) * SZ + ci] = (Real)(jxw * b0);
        W[(el * 3 + 1) * SZ + ci] = (Real)(jxw * b1);
        W[(el * 3 + 2) * SZ + ci] = (Real)(jxw * b2);
    }
    __syncthreads();
    sweep<Real, 2, TB, true, false, 1, 0, 1, 0>(W, U, 3 * EPB);
    __syncthreads();
    sweep<Real, 1, TB, true, false, 1, 0, 1, 0>(U, W, 3 * EPB);
    __syncthreads();
    sweep<Real, 0, TB, true, false, 1, 0, 1, 0>(W, U, 3 * EPB);
    __syncthreads();
    scatter_add(m, e0, EPB, U, f, true);
}

// geometry at every quadrature point: J0 = dX/dxi from the degree-g map,
// J0^-1 (row-major (J0^-1)_{ed}) and JxW = det J0 * w (FP64 and FP32 copies)
__global__ void __launch_bounds__(256) k_geometry(const hx::MeshView m, const double *__restrict__ X, const int32_t *__restrict__ gconn,
                           int g, double *__restrict__ geo64, float *__restrict__ geo32) {
    const int ng = g + 1, ngg = ng * ng * ng;
    const int64_t total = m.n_qp;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(idx / NQ);
        const int q = (int)(idx - (int64_t)e * NQ);
        const int qx = q % N, qy = (q / N) % N, qz = q / NN;
        double J0[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int a = 0; a < ngg; ++a) {
            const int ia = a % ng, ja = (a / ng) % ng, ka = a / (ng * ng);
            const double vx = cGeoV[g - 1][ia * N + qx], vy = cGeoV[g - 1][ja * N + qy], vz = cGeoV[g - 1][ka * N + qz];
            const double dx = cGeoD[g - 1][ia * N + qx], dy = cGeoD[g - 1][ja * N + qy], dz = cGeoD[g - 1][ka * N + qz];
            const double d0 = dx * vy * vz, d1 = vx * dy * vz, d2 = vx * vy * dz;
            const double *xp = X + 3 * (int64_t)gconn[(int64_t)e * ngg + a];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                J0[r * 3 + 0] += xp[r] * d0;
                J0[r * 3 + 1] += xp[r] * d1;
                J0[r * 3 + 2] += xp[r] * d2;
            }
        }
        const double det = J0[0] * (J0[4] * J0[8] - J0[5] * J0[7]) - J0[1] * (J0[3] * J0[8] - J0[5] * J0[6]) +
                           J0[2] * (J0[3] * J0[7] - J0[4] * J0[6]);
        if (!(det > 0.0)) atomicOr(m.err + 0, 2);
        const double id = 1.0 / det;
        double Ji[9];
        Ji[0] = (J0[4] * J0[8] - J0[5] * J0[7]) * id;
        Ji[1] = (J0[2] * J0[7] - J0[1] * J0[8]) * id;
        Ji[2] = (J0[1] * J0[5] - J0[2] * J0[4]) * id;
        Ji[3] = (J0[5] * J0[6] - J0[3] * J0[8]) * id;
        Ji[4] = (J0[0] * J0[8] - J0[2] * J0[6]) * id;
        Ji[5] = (J0[2] * J0[3] - J0[0] * J0[5]) * id;
        Ji[6] = (J0[3] * J0[7] - J0[4] * J0[6]) * id;
        Ji[7] = (J0[1] * J0[6] - J0[0] * J0[7]) * id;
        Ji[8] = (J0[0] * J0[4] - J0[1] * J0[3]) * id;
        const double jxw = det * cW[qx] * cW[qy] * cW[qz];
        for (int k = 0; k < 9; ++k) {
            geo64[(int64_t)k * m.qs + idx] = Ji[k];
            geo32[(int64_t)k * m.qs + idx] = (float)Ji[k];
        }
        geo64[(int64_t)9 * m.qs + idx] = jxw;
        geo32[(int64_t)9 * m.qs + idx] = (float)jxw;
    }
}

__global__ void __launch_bounds__(256) k_node_coords(const hx::MeshView m, const double *__restrict__ X, const int32_t *__restrict__ gconn,
                              int g, double *__restrict__ out) {
    const int ng = g + 1, ngg = ng * ng * ng;
    const int64_t total = (int64_t)m.n_elem * NQ;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(idx / NQ);
        const int a = (int)(idx - (int64_t)e * NQ);
        const int i = a % N, j = (a / N) % N, k = a / NN;
        double x[3] = {0, 0, 0};
        for (int b = 0; b < ngg; ++b) {
            const int ib = b % ng, jb = (b / ng) % ng, kb = b / (ng * ng);
            const double w = cGeoVn[g - 1][ib * N + i] * cGeoVn[g - 1][jb * N + j] * cGeoVn[g - 1][kb * N + k];
            const double *xp = X + 3 * (int64_t)gconn[(int64_t)e * ngg + b];
            x[0] += w * xp[0];
            x[1] += w * xp[1];
            x[2] += w * xp[2];
        }
        const int64_t nd = node_of(m, e, i, j, k);
        out[3 * nd + 0] = x[0];
        out[3 * nd + 1] = x[1];
        out[3 * nd + 2] = x[2];
    }
}

__global__ void k_convert_uk(const double *__restrict__ u, Real *__restrict__ uk, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        uk[i] = (Real)u[i];
}

// copy the 1D tables of this degree into this unit's constant memory
cudaError_t op_upload(const double *B, const double *D, const double *Gd, const double *w, const double *geoV,
                      const double *geoD, const double *geoVn) {
    Real t[3][NN];
    for (int i = 0; i < NN; ++i) {
        t[0][i] = (Real)B[i];
        t[1][i] = (Real)D[i];
        t[2][i] = (Real)Gd[i];
    }
    cudaError_t e = cudaMemcpyToSymbol(cTab, t, sizeof t);
    if (PK && e == cudaSuccess) {  // {m, m} pairs for the paired sweeps
        float2 t2[3][NN];
        for (int k = 0; k < 3; ++k)
            for (int i = 0; i < NN; ++i) t2[k][i] = make_float2((float)t[k][i], (float)t[k][i]);
        e = cudaMemcpyToSymbol(cTab2, t2, sizeof t2);
    }
    if (EOH > 0) {
        Real eo[3][2][2][(EOH > 0 ? EOH : 1) * (EOH > 0 ? EOH : 1)];
        const double *src[3] = {B, D, Gd};
        for (int k = 0; k < 3; ++k)
            for (int tr = 0; tr < 2; ++tr)
                for (int o = 0; o < EOH; ++o)
                    for (int c = 0; c < EOH; ++c) {
                        auto Mx = [&](int r, int q) { return tr ? src[k][q * N + r] : src[k][r * N + q]; };
                        eo[k][tr][0][o * EOH + c] = (Real)(0.5 * (Mx(o, c) + Mx(o, N - 1 - c)));
                        eo[k][tr][1][o * EOH + c] = (Real)(0.5 * (Mx(o, c) - Mx(o, N - 1 - c)));
                    }
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(cEO, eo, sizeof eo);
        if (PK && e == cudaSuccess) {
            float2 eo2[3][2][2][(EOH > 0 ? EOH : 1) * (EOH > 0 ? EOH : 1)];
            for (int k = 0; k < 3; ++k)
                for (int tr = 0; tr < 2; ++tr)
                    for (int h = 0; h < 2; ++h)
                        for (int i = 0; i < EOH * EOH; ++i)
                            eo2[k][tr][h][i] = make_float2((float)eo[k][tr][h][i], (float)eo[k][tr][h][i]);
            e = cudaMemcpyToSymbol(cEO2, eo2, sizeof eo2);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cW, w, sizeof(double) * N);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cGeoV, geoV, sizeof(double) * 2 * 3 * N);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cGeoD, geoD, sizeof(double) * 2 * 3 * N);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cGeoVn, geoVn, sizeof(double) * 2 * 3 * N);
    return e;
}
