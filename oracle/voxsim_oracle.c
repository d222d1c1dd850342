/*
 * voxsim_oracle.c -- plain FP64 CPU oracle of the voxel soft-robot co-design hot path of
 * "CUDA-Accelerated Soft Robot Neural Evolution with Large Language Model Supervision"
 * (L. Zhang, arXiv 2405.00698).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, plain definition that the CUDA library is checked
 * against.  Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or helper with the CUDA library, and it never
 * receives an input produced by the CUDA path.
 *
 * Every step is written in the order the method states it, over plain loops, in double
 * precision.  Where the paper fixes nothing (integrator, force law, friction, fitness, the
 * evolutionary operators' random numbers) the function comment states the reading taken.
 *
 * Parity pins live in the pytest suite (closed forms, invariants, library routines, brute
 * force).  The only part without an external pin is the long-horizon agreement of chaotic
 * contact trajectories: "parity unpinned" for trajectories beyond the 1000-step horizon.
 *
 * Material ids (Section II-A): 0 empty, 1 expanding muscle, 2 contracting muscle,
 * 3 soft tissue, 4 bone.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_NMAT 5

/* Physics and material constants (Table II, plus the configuration values that override it).
 * Layout mirrored by the ctypes structure in oracle.py. */
typedef struct {
    double dt;          /* time step [s] */
    double gravity;     /* [m/s^2] */
    double mass;        /* point mass per voxel corner [kg] */
    double edge;        /* voxel edge = original rest length [m] */
    double damping;     /* velocity multiplier per step (1 = none) */
    double k_ground;    /* ground penalty stiffness [N/m] */
    double mu_s;        /* static friction coefficient */
    double mu_k;        /* kinetic friction coefficient */
    double freq;        /* muscle actuation frequency [Hz] */
    double dead_bound;  /* |coordinate| beyond this marks the robot dead [m] */
    double k_mat[ORC_NMAT];     /* stiffness per material [N/m] */
    double amp_mat[ORC_NMAT];   /* actuation amplitude per material (fraction of L0) */
    double phase_mat[ORC_NMAT]; /* actuation phase per material [rad] */
    int32_t ground_on;  /* 0 disables the ground (conservation pins) */
    int32_t pad_;
    double spring_zeta; /* spring dashpot damping ratio (Table II; 0 in the configurations) */
    double ground_zeta; /* ground damping ratio (Table II; 0 in the configurations) */
} orc_params;

/* ------------------------------------------------------------------------------------------ */
/* Gaussian positional encoding and the MLP spatial query (Eq. (1), Section II-B/II-C).        */
/* ------------------------------------------------------------------------------------------ */

/* Round a double to the nearest bfloat16 value (ties to even), returned as a double.
 * bfloat16 keeps the float32 exponent and 8 significant bits (7 stored). */
double orc_round_bf16(double x)
{
    if (x == 0.0 || isnan(x) || isinf(x)) return x;
    int e;
    double m = frexp(fabs(x), &e);          /* |x| = m * 2^e, m in [0.5, 1) */
    if (e < -125) {                          /* subnormal bf16 range: fixed quantum 2^-133 */
        double q = ldexp(1.0, -133);
        double r = nearbyint(fabs(x) / q) * q;  /* default rounding mode: ties to even */
        return copysign(r, x);
    }
    double scaled = ldexp(m, 8);             /* 8 significant bits -> integer part */
    double r = nearbyint(scaled);            /* ties to even */
    double out = ldexp(r, e - 8);
    if (out > 3.38953138925153547590e38) out = INFINITY; /* above the bf16 maximum */
    return copysign(out, x);
}

/* Genome layout of the MLP 3 -> gamma(256) -> 64 -> 64 -> 6: W1[64][256], b1[64], W2[64][64],
 * b2[64], W3[6][64], b3[6]; 20998 float32 values.  Output 0..4 are the material scores (softmax
 * branch), output 5 the material weight (sigmoid branch). */
enum { ORC_PE_M = 128, ORC_PE_D = 256, ORC_H = 64, ORC_OUT = 6,
       ORC_OFF_W1 = 0, ORC_OFF_B1 = 16384, ORC_OFF_W2 = 16448, ORC_OFF_B2 = 20544,
       ORC_OFF_W3 = 20608, ORC_OFF_B3 = 20992, ORC_GENOME = 20998 };

/* Eq. (1): gamma(v) = [cos(2 pi B v), sin(2 pi B v)] at the voxel centre
 * v = ((i+1/2)/nx, (j+1/2)/ny, (k+1/2)/nz); B is m x 3 (m = 128), cos block first.
 * out[q*256 + c] for query q = i + nx*(j + ny*k).  Values are exact doubles (no rounding). */
void orc_pe_table(int nx, int ny, int nz, const float* B, double* out)
{
    const double two_pi = 2.0 * M_PI;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int q = i + nx * (j + ny * k);
                double v0 = (i + 0.5) / nx, v1 = (j + 0.5) / ny, v2 = (k + 0.5) / nz;
                for (int r = 0; r < ORC_PE_M; ++r) {
                    double bv = (double)B[3 * r + 0] * v0;
                    bv = bv + (double)B[3 * r + 1] * v1;
                    bv = bv + (double)B[3 * r + 2] * v2;
                    double arg = two_pi * bv;
                    out[(size_t)q * ORC_PE_D + r] = cos(arg);
                    out[(size_t)q * ORC_PE_D + ORC_PE_M + r] = sin(arg);
                }
            }
}

/* MLP spatial query of one genome over a whole grid (Section II-C, Fig. 1).
 * The tensor-core path rounds its operands to bfloat16: gamma, W1, W2, W3 and the hidden
 * activations h1, h2.  The oracle rounds at the same points and accumulates in double.
 * Biases stay float32.  Outputs per query: the six raw outputs (logits_out, optional), the
 * chosen material = argmax of the five scores taken on the float32-rounded scores (softmax is
 * monotone, so it does not change the choice; ties go to the lowest material id), the material
 * weight w = sigmoid(o5), and a guard band (guard_out, optional) on how far a float32
 * implementation with the same rounding points can move the six outputs.  A float32 sum of K
 * terms differs from the exact one by at most delta = 2 (K + 2) 2^-24 sum |terms|; a hidden
 * activation h = bf16(relu(x)) can then change only if bf16(relu(x - delta)) differs from
 * bf16(relu(x + delta)), by at most that difference.  The bound is carried through the layers
 * (a changed h1 widens the next layer's delta by |W2| times its change) and the guard is the
 * largest output bound. */
static double relu_bf16(double x) { return orc_round_bf16(x > 0.0 ? x : 0.0); }

static double acc_err(int K, double mag) { return 2.0 * (K + 2) * ldexp(mag, -24); }

void orc_mlp_query(int nx, int ny, int nz, const float* B, const float* genome,
                   uint8_t* mat_out, double* w_out, double* logits_out, double* guard_out)
{
    int Q = nx * ny * nz;
    double* pe = (double*)malloc(sizeof(double) * (size_t)Q * ORC_PE_D);
    orc_pe_table(nx, ny, nz, B, pe);
    const float* W1 = genome + ORC_OFF_W1; const float* b1 = genome + ORC_OFF_B1;
    const float* W2 = genome + ORC_OFF_W2; const float* b2 = genome + ORC_OFF_B2;
    const float* W3 = genome + ORC_OFF_W3; const float* b3 = genome + ORC_OFF_B3;
    double g[ORC_PE_D], h1[ORC_H], h2[ORC_H], o[ORC_OUT];
    for (int q = 0; q < Q; ++q) {
        for (int c = 0; c < ORC_PE_D; ++c) g[c] = orc_round_bf16(pe[(size_t)q * ORC_PE_D + c]);
        double dh1[ORC_H], dh2[ORC_H];
        for (int r = 0; r < ORC_H; ++r) {
            double acc = 0.0, mag = 0.0;
            for (int c = 0; c < ORC_PE_D; ++c) {
                double t = orc_round_bf16(W1[r * ORC_PE_D + c]) * g[c];
                acc += t;
                mag += fabs(t);
            }
            acc += (double)b1[r];
            mag += fabs((double)b1[r]);
            h1[r] = relu_bf16(acc);
            double d = acc_err(ORC_PE_D, mag);
            dh1[r] = fabs(relu_bf16(acc + d) - relu_bf16(acc - d));
        }
        for (int r = 0; r < ORC_H; ++r) {
            double acc = 0.0, mag = 0.0, prop = 0.0;
            for (int c = 0; c < ORC_H; ++c) {
                double wq = orc_round_bf16(W2[r * ORC_H + c]);
                acc += wq * h1[c];
                mag += fabs(wq * h1[c]);
                prop += fabs(wq) * dh1[c];
            }
            acc += (double)b2[r];
            mag += fabs((double)b2[r]);
            h2[r] = relu_bf16(acc);
            double d = prop + acc_err(ORC_H, mag);
            dh2[r] = fabs(relu_bf16(acc + d) - relu_bf16(acc - d));
        }
        double spread = 0.0;
        for (int r = 0; r < ORC_OUT; ++r) {
            double acc = 0.0, mag = 0.0, prop = 0.0;
            for (int c = 0; c < ORC_H; ++c) {
                double wq = orc_round_bf16(W3[r * ORC_H + c]);
                acc += wq * h2[c];
                mag += fabs(wq * h2[c]);
                prop += fabs(wq) * dh2[c];
            }
            o[r] = acc + (double)b3[r];
            double bound = prop + acc_err(ORC_H, mag + fabs((double)b3[r]));
            if (bound > spread) spread = bound;
        }
        int best = 0;
        float bestv = (float)o[0];
        for (int c = 1; c < 5; ++c)
            if ((float)o[c] > bestv) { bestv = (float)o[c]; best = c; }
        mat_out[q] = (uint8_t)best;
        w_out[q] = 1.0 / (1.0 + exp(-o[5]));
        if (logits_out) for (int r = 0; r < ORC_OUT; ++r) logits_out[(size_t)q * ORC_OUT + r] = o[r];
        if (guard_out) guard_out[q] = spread;
    }
    free(pe);
}

/* ------------------------------------------------------------------------------------------ */
/* Largest connected component (6-connectivity).                                                */
/* ------------------------------------------------------------------------------------------ */

/* Keep only the largest face-connected component of occupied voxels (material != 0).
 * Components are found by breadth-first search started from voxels in increasing linear index
 * i + nx*(j + ny*k); a component therefore carries its smallest index as its discovery order,
 * and a size tie keeps the component discovered first.  Returns the kept voxel count. */
int orc_lcc_bfs(int nx, int ny, int nz, const uint8_t* mat_in, uint8_t* mat_out)
{
    int V = nx * ny * nz;
    int* comp = (int*)malloc(sizeof(int) * (size_t)(V > 0 ? V : 1));
    int* queue = (int*)malloc(sizeof(int) * (size_t)(V > 0 ? V : 1));
    for (int v = 0; v < V; ++v) comp[v] = -1;
    int ncomp = 0, best = -1, best_size = 0;
    for (int s = 0; s < V; ++s) {
        if (mat_in[s] == 0 || comp[s] >= 0) continue;
        int head = 0, tail = 0, size = 0;
        queue[tail++] = s;
        comp[s] = ncomp;
        while (head < tail) {
            int v = queue[head++];
            ++size;
            int i = v % nx, j = (v / nx) % ny, k = v / (nx * ny);
            int nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k},
                            {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
            for (int t = 0; t < 6; ++t) {
                int a = nb[t][0], b = nb[t][1], c = nb[t][2];
                if (a < 0 || b < 0 || c < 0 || a >= nx || b >= ny || c >= nz) continue;
                int u = a + nx * (b + ny * c);
                if (mat_in[u] != 0 && comp[u] < 0) { comp[u] = ncomp; queue[tail++] = u; }
            }
        }
        if (size > best_size) { best_size = size; best = ncomp; }
        ++ncomp;
    }
    for (int v = 0; v < V; ++v) mat_out[v] = (best >= 0 && comp[v] == best) ? mat_in[v] : 0;
    free(comp);
    free(queue);
    return best_size;
}

static int uf_find(int* parent, int x)
{
    while (parent[x] != x) x = parent[x];
    return x;
}

/* Second, independent largest-component routine (union-find with smallest-index roots), used
 * only to cross-check the breadth-first version above. */
int orc_lcc_unionfind(int nx, int ny, int nz, const uint8_t* mat_in, uint8_t* mat_out)
{
    int V = nx * ny * nz;
    int* parent = (int*)malloc(sizeof(int) * (size_t)(V > 0 ? V : 1));
    int* size = (int*)calloc((size_t)(V > 0 ? V : 1), sizeof(int));
    for (int v = 0; v < V; ++v) parent[v] = v;
    for (int v = 0; v < V; ++v) {
        if (mat_in[v] == 0) continue;
        int i = v % nx, j = (v / nx) % ny, k = v / (nx * ny);
        int fwd[3] = {i + 1 < nx ? v + 1 : -1, j + 1 < ny ? v + nx : -1,
                      k + 1 < nz ? v + nx * ny : -1};
        for (int t = 0; t < 3; ++t) {
            int u = fwd[t];
            if (u < 0 || mat_in[u] == 0) continue;
            int ra = uf_find(parent, v), rb = uf_find(parent, u);
            if (ra == rb) continue;
            if (ra < rb) parent[rb] = ra; else parent[ra] = rb;
        }
    }
    for (int v = 0; v < V; ++v)
        if (mat_in[v] != 0) size[uf_find(parent, v)]++;
    int best = -1, best_size = 0;
    for (int v = 0; v < V; ++v)   /* roots are the smallest index of their component */
        if (size[v] > best_size) { best_size = size[v]; best = v; }
    for (int v = 0; v < V; ++v)
        mat_out[v] = (mat_in[v] != 0 && uf_find(parent, v) == best) ? mat_in[v] : 0;
    free(parent);
    free(size);
    return best_size;
}

/* ------------------------------------------------------------------------------------------ */
/* Robot: topology, parameters, state.                                                          */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int nx, ny, nz, V;
    uint8_t* mat;           /* per voxel, after the largest-component filter */
    double *w, *kappa, *phi;/* per voxel material weight, stiffness, actuation phase */
    int M;                  /* masses */
    int* mass_corner;       /* corner id c = ci + (nx+1)*(cj + (ny+1)*ck), ascending */
    int* corner_mass;       /* inverse map, -1 where no mass */
    int S;                  /* springs */
    int *sa, *sb;           /* endpoints (mass indices), sa < sb, sorted by (sa, sb) */
    int* s_ninc;            /* number of incident kept voxels */
    int* s_vox;             /* up to 4 incident voxel ids per spring (-1 padded) */
    double *L0, *ks, *alpha, *beta; /* rest length, stiffness, actuation sin / cos coefficients */
    double *x, *v;          /* M*3 state */
    double x0_centroid;     /* mean x of the initial pose */
    long step;              /* global step counter of this robot */
} orc_robot;

typedef struct { int a, b, vox; } orc_triple;

static int cmp_triple(const void* p, const void* q)
{
    const orc_triple* s = (const orc_triple*)p; const orc_triple* t = (const orc_triple*)q;
    if (s->a != t->a) return s->a < t->a ? -1 : 1;
    if (s->b != t->b) return s->b < t->b ? -1 : 1;
    return (s->vox > t->vox) - (s->vox < t->vox);
}

/* Per-spring stiffness and actuation coefficients from the per-voxel parameters.
 * A voxel contributes k_v = w_v * kappa_v and the actuation a_v sin(w t + phi_v) with
 * a_v = w_v * amp_mat[material]; a spring shared by several kept voxels takes the mean over them:
 * k_s = mean k_v, and mean a_v sin(w t + phi_v) = alpha_s sin(w t) + beta_s cos(w t) with
 * alpha_s = mean a_v cos(phi_v), beta_s = mean a_v sin(phi_v). */
static void orc_spring_params(orc_robot* R, const orc_params* p)
{
    for (int s = 0; s < R->S; ++s) {
        double ksum = 0.0, asum = 0.0, bsum = 0.0;
        int n = R->s_ninc[s];
        for (int t = 0; t < n; ++t) {
            int v = R->s_vox[4 * s + t];
            double amp = R->w[v] * p->amp_mat[R->mat[v]];
            ksum += R->w[v] * R->kappa[v];
            asum += amp * cos(R->phi[v]);
            bsum += amp * sin(R->phi[v]);
        }
        R->ks[s] = ksum / n;
        R->alpha[s] = asum / n;
        R->beta[s] = bsum / n;
    }
}

/* Build a robot from its decoded voxel grid (Section II-A; Table II).
 * Masses sit at the corners of kept voxels, ordered by ascending corner id.  Springs join all 28
 * corner pairs of every kept voxel; a pair shared by several voxels is one spring.  Rest length
 * is the lattice distance (edge * {1, sqrt 2, sqrt 3}).  The initial pose is the lattice itself
 * shifted so the lowest mass sits at z = 0, at rest.  w, kappa, phi may be NULL: then w = 1,
 * kappa = k_mat[material], phi = phase_mat[material].  If apply_lcc, the largest-component filter
 * runs first. */
orc_robot* orc_robot_new(int nx, int ny, int nz, const uint8_t* mat_in, const double* w,
                         const double* kappa, const double* phi, const orc_params* p,
                         int apply_lcc)
{
    orc_robot* R = (orc_robot*)calloc(1, sizeof(orc_robot));
    R->nx = nx; R->ny = ny; R->nz = nz; R->V = nx * ny * nz;
    int V = R->V;
    R->mat = (uint8_t*)malloc((size_t)(V > 0 ? V : 1));
    if (apply_lcc) orc_lcc_bfs(nx, ny, nz, mat_in, R->mat);
    else memcpy(R->mat, mat_in, (size_t)V);
    R->w = (double*)malloc(sizeof(double) * (size_t)(V > 0 ? V : 1));
    R->kappa = (double*)malloc(sizeof(double) * (size_t)(V > 0 ? V : 1));
    R->phi = (double*)malloc(sizeof(double) * (size_t)(V > 0 ? V : 1));
    for (int v = 0; v < V; ++v) {
        int m = R->mat[v];
        R->w[v] = w ? w[v] : 1.0;
        R->kappa[v] = kappa ? kappa[v] : p->k_mat[m];
        R->phi[v] = phi ? phi[v] : p->phase_mat[m];
    }
    int cx = nx + 1, cy = ny + 1, cz = nz + 1, C = cx * cy * cz;
    R->corner_mass = (int*)malloc(sizeof(int) * (size_t)C);
    for (int c = 0; c < C; ++c) R->corner_mass[c] = -1;
    /* corners of kept voxels */
    char* used = (char*)calloc((size_t)C, 1);
    for (int k = 0; k < nz; ++k) for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
        if (R->mat[i + nx * (j + ny * k)] == 0) continue;
        for (int d = 0; d < 8; ++d) {
            int a = i + (d & 1), b = j + ((d >> 1) & 1), c = k + ((d >> 2) & 1);
            used[a + cx * (b + cy * c)] = 1;
        }
    }
    int M = 0;
    for (int c = 0; c < C; ++c) if (used[c]) ++M;
    R->M = M;
    R->mass_corner = (int*)malloc(sizeof(int) * (size_t)(M > 0 ? M : 1));
    M = 0;
    for (int c = 0; c < C; ++c) if (used[c]) { R->corner_mass[c] = M; R->mass_corner[M++] = c; }
    free(used);
    /* all (corner pair, voxel) incidences, then sorted and grouped into unique springs */
    int nkept = 0;
    for (int v = 0; v < V; ++v) if (R->mat[v]) ++nkept;
    orc_triple* tr = (orc_triple*)malloc(sizeof(orc_triple) * (size_t)(28 * nkept + 1));
    int nt = 0;
    for (int k = 0; k < nz; ++k) for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
        int v = i + nx * (j + ny * k);
        if (R->mat[v] == 0) continue;
        int cm[8];
        for (int d = 0; d < 8; ++d) {
            int a = i + (d & 1), b = j + ((d >> 1) & 1), c = k + ((d >> 2) & 1);
            cm[d] = R->corner_mass[a + cx * (b + cy * c)];
        }
        for (int d = 0; d < 8; ++d)
            for (int e = d + 1; e < 8; ++e) {
                int a = cm[d], b = cm[e];
                tr[nt].a = a < b ? a : b; tr[nt].b = a < b ? b : a; tr[nt].vox = v; ++nt;
            }
    }
    qsort(tr, (size_t)nt, sizeof(orc_triple), cmp_triple);
    int S = 0;
    for (int t = 0; t < nt; ++t)
        if (t == 0 || tr[t].a != tr[t - 1].a || tr[t].b != tr[t - 1].b) ++S;
    R->S = S;
    size_t sc = (size_t)(S > 0 ? S : 1);
    R->sa = (int*)malloc(sizeof(int) * sc); R->sb = (int*)malloc(sizeof(int) * sc);
    R->s_ninc = (int*)calloc(sc, sizeof(int)); R->s_vox = (int*)malloc(sizeof(int) * 4 * sc);
    R->L0 = (double*)malloc(sizeof(double) * sc); R->ks = (double*)malloc(sizeof(double) * sc);
    R->alpha = (double*)malloc(sizeof(double) * sc); R->beta = (double*)malloc(sizeof(double) * sc);
    for (size_t s = 0; s < 4 * sc; ++s) R->s_vox[s] = -1;
    int s = -1;
    for (int t = 0; t < nt; ++t) {
        if (t == 0 || tr[t].a != tr[t - 1].a || tr[t].b != tr[t - 1].b) {
            ++s;
            R->sa[s] = tr[t].a; R->sb[s] = tr[t].b;
        }
        R->s_vox[4 * s + R->s_ninc[s]] = tr[t].vox;
        R->s_ninc[s]++;
    }
    free(tr);
    /* initial pose: lattice, lowest corner at z = 0 */
    R->x = (double*)malloc(sizeof(double) * 3 * (size_t)(M > 0 ? M : 1));
    R->v = (double*)calloc(3 * (size_t)(M > 0 ? M : 1), sizeof(double));
    int zmin = cz;
    for (int m = 0; m < M; ++m) {
        int c = R->mass_corner[m];
        int ck = c / (cx * cy);
        if (ck < zmin) zmin = ck;
    }
    double xsum = 0.0;
    for (int m = 0; m < M; ++m) {
        int c = R->mass_corner[m];
        int ci = c % cx, cj = (c / cx) % cy, ck = c / (cx * cy);
        R->x[3 * m + 0] = ci * p->edge;
        R->x[3 * m + 1] = cj * p->edge;
        R->x[3 * m + 2] = (ck - zmin) * p->edge;
        xsum += R->x[3 * m + 0];
    }
    R->x0_centroid = M > 0 ? xsum / M : 0.0;
    for (int q = 0; q < S; ++q) {
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = R->x[3 * R->sb[q] + a] - R->x[3 * R->sa[q] + a];
        R->L0[q] = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
    orc_spring_params(R, p);
    R->step = 0;
    return R;
}

void orc_robot_free(orc_robot* R)
{
    if (!R) return;
    free(R->mat); free(R->w); free(R->kappa); free(R->phi);
    free(R->mass_corner); free(R->corner_mass);
    free(R->sa); free(R->sb); free(R->s_ninc); free(R->s_vox);
    free(R->L0); free(R->ks); free(R->alpha); free(R->beta);
    free(R->x); free(R->v);
    free(R);
}

void orc_robot_counts(const orc_robot* R, int32_t* M, int32_t* S)
{
    *M = R->M;
    *S = R->S;
}

/* Copy out topology and per-spring parameters (arrays sized by orc_robot_counts). */
void orc_robot_topology(const orc_robot* R, uint8_t* kept_mat, int32_t* mass_corner,
                        int32_t* spring_a, int32_t* spring_b, double* L0, double* k,
                        double* alpha, double* beta)
{
    if (kept_mat) memcpy(kept_mat, R->mat, (size_t)R->V);
    for (int m = 0; m < R->M; ++m) if (mass_corner) mass_corner[m] = R->mass_corner[m];
    for (int s = 0; s < R->S; ++s) {
        if (spring_a) spring_a[s] = R->sa[s];
        if (spring_b) spring_b[s] = R->sb[s];
        if (L0) L0[s] = R->L0[s];
        if (k) k[s] = R->ks[s];
        if (alpha) alpha[s] = R->alpha[s];
        if (beta) beta[s] = R->beta[s];
    }
}

void orc_robot_get_state(const orc_robot* R, double* x, double* v)
{
    if (x) memcpy(x, R->x, sizeof(double) * 3 * (size_t)R->M);
    if (v) memcpy(v, R->v, sizeof(double) * 3 * (size_t)R->M);
}

void orc_robot_set_state(orc_robot* R, const double* x, const double* v, long step)
{
    if (x) memcpy(R->x, x, sizeof(double) * 3 * (size_t)R->M);
    if (v) memcpy(R->v, v, sizeof(double) * 3 * (size_t)R->M);
    R->step = step;
}

/* ------------------------------------------------------------------------------------------ */
/* Time stepping (Section II-C: per-spring and per-mass updates; Table II constants).           */
/* ------------------------------------------------------------------------------------------ */

/* Contact mode of one mass in one step: 0 no contact, 1 stick, 2 slip, 3 slip with the kinetic
 * friction saturated (mu_k F_n >= |F_h|: the horizontal force is cancelled, the velocity kept). */
enum { ORC_FREE = 0, ORC_STICK = 1, ORC_SLIP = 2, ORC_SLIP_HELD = 3 };

/* One time step of one robot at time t = step * dt.
 *  1. every mass starts from its weight (0, 0, -m g);
 *  2. every spring s = (a, b): d = x_b - x_a, l = |d|, actuated rest length
 *     L = L0 (1 + alpha_s sin(w t) + beta_s cos(w t)) with w = 2 pi freq; Hooke force
 *     f = k_s (l - L) d / l is added to mass a and subtracted from mass b;
 *     With a spring damping ratio zeta_s > 0 (Table II; the paper's own preset), a dashpot
 *     c_s ((v_b - v_a) . u) u with c_s = 2 zeta_s sqrt(k_s m / 2) (the critical damping of two
 *     equal masses) is added to the spring force;
 *  3. every mass below the ground plane (z < 0) gets the penalty normal force
 *     F_n = k_ground (-z) added to F_z (and, with a ground damping ratio zeta_g > 0, the dashpot
 *     -2 zeta_g sqrt(k_ground m) v_z); with F_h = (F_x, F_y): if |F_h| <= mu_s F_n the mass
 *     sticks (F_h = 0 and horizontal velocity = 0), otherwise it slips and kinetic friction
 *     mu_k F_n is removed along F_h, never more than |F_h| itself: Table II prints
 *     mu_s = 0.6 < mu_k = 1.0, and with mu_s F_n < |F_h| < mu_k F_n the full kinetic term would
 *     reverse the horizontal force; the reading taken is that friction at most cancels it
 *     (mode 3: F_h = 0, the velocity kept);
 *  4. semi-implicit Euler with velocity damping: v <- c (v + dt F / m), x <- x + dt v.
 * modes (optional, M entries) records the contact mode of every mass and Fpre (optional, 3M)
 * the force before the contact step.  force (optional, M entries) imposes the contact mode of
 * every mass instead of deciding it from the state: free adds no ground force; stick and slip
 * add F_n = k_ground (-z) whatever the sign of z and then zero the horizontal force and velocity
 * (stick), remove mu_k F_n along F_h (slip) or zero the horizontal force only (saturated slip)
 * -- the same piecewise formulas, selected from outside (used to difference the step map along another run's contact decisions).  Returns the
 * number of springs skipped for zero length. */
static int orc_step(orc_robot* R, const orc_params* p, double* F, uint8_t* modes, double* Fpre,
                    const uint8_t* force)
{
    const double t = (double)R->step * p->dt;
    const double wt = 2.0 * M_PI * p->freq * t;
    const double sn = sin(wt), cs = cos(wt);
    int M = R->M, skipped = 0;
    for (int m = 0; m < M; ++m) {
        F[3 * m + 0] = 0.0; F[3 * m + 1] = 0.0; F[3 * m + 2] = -p->mass * p->gravity;
    }
    for (int s = 0; s < R->S; ++s) {
        int a = R->sa[s], b = R->sb[s];
        double d[3];
        for (int q = 0; q < 3; ++q) d[q] = R->x[3 * b + q] - R->x[3 * a + q];
        double l = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (l < 1e-12) { ++skipped; continue; }
        double L = R->L0[s] * (1.0 + R->alpha[s] * sn + R->beta[s] * cs);
        double fm = R->ks[s] * (l - L) / l;
        if (p->spring_zeta > 0.0) {
            /* dashpot along the spring: c_s ((v_b - v_a) . u) u, c_s = 2 zeta sqrt(k_s m / 2) */
            double cs_ = 2.0 * p->spring_zeta * sqrt(R->ks[s] * p->mass / 2.0);
            double rv = 0.0;
            for (int q = 0; q < 3; ++q) rv += (R->v[3 * b + q] - R->v[3 * a + q]) * d[q] / l;
            fm += cs_ * rv / l;
        }
        for (int q = 0; q < 3; ++q) { F[3 * a + q] += fm * d[q]; F[3 * b + q] -= fm * d[q]; }
    }
    if (Fpre) memcpy(Fpre, F, sizeof(double) * 3 * (size_t)M);
    for (int m = 0; m < M; ++m) {
        double* x = R->x + 3 * m; double* v = R->v + 3 * m; double* f = F + 3 * m;
        uint8_t mode = ORC_FREE;
        const int contact = force ? force[m] != ORC_FREE : (p->ground_on && x[2] < 0.0);
        if (contact) {
            double fn = p->k_ground * (-x[2]);
            f[2] += fn;
            /* ground dashpot on the normal velocity: c_g = 2 zeta sqrt(k_g m) */
            if (p->ground_zeta > 0.0) f[2] -= 2.0 * p->ground_zeta * sqrt(p->k_ground * p->mass) * v[2];
            double fh = sqrt(f[0] * f[0] + f[1] * f[1]);
            if (force ? force[m] == ORC_STICK : fh <= p->mu_s * fn) {
                mode = ORC_STICK;
                f[0] = 0.0; f[1] = 0.0; v[0] = 0.0; v[1] = 0.0;
            } else if (force ? force[m] == ORC_SLIP_HELD : p->mu_k * fn >= fh) {
                mode = ORC_SLIP_HELD;             /* kinetic friction cancels F_h exactly */
                f[0] = 0.0; f[1] = 0.0;
            } else {
                mode = ORC_SLIP;
                double scale = 1.0 - p->mu_k * fn / fh;
                f[0] *= scale; f[1] *= scale;
            }
        }
        if (modes) modes[m] = mode;
        for (int q = 0; q < 3; ++q) {
            v[q] = p->damping * (v[q] + p->dt * f[q] / p->mass);
            x[q] = x[q] + p->dt * v[q];
        }
    }
    R->step++;
    return skipped;
}

/* Advance one robot by nsteps.  Returns the number of zero-length spring skips. */
int orc_robot_simulate(orc_robot* R, const orc_params* p, int nsteps)
{
    double* F = (double*)malloc(sizeof(double) * 3 * (size_t)(R->M > 0 ? R->M : 1));
    int skipped = 0;
    for (int n = 0; n < nsteps; ++n) skipped += orc_step(R, p, F, NULL, NULL, NULL);
    free(F);
    return skipped;
}

/* Advance one robot by nsteps with the contact modes of every step imposed (force: nsteps x M in
 * mass order, see orc_step).  Returns the number of zero-length spring skips. */
int orc_robot_simulate_modes(orc_robot* R, const orc_params* p, int nsteps, const uint8_t* force)
{
    double* F = (double*)malloc(sizeof(double) * 3 * (size_t)(R->M > 0 ? R->M : 1));
    int skipped = 0;
    for (int n = 0; n < nsteps; ++n)
        skipped += orc_step(R, p, F, NULL, NULL, force + (size_t)n * (size_t)R->M);
    free(F);
    return skipped;
}

/* Fitness: displacement of the centroid along +x, final minus initial pose, equal masses.
 * The paper only names "fitness" (Section III); the centroid x-displacement is the reading taken.
 * An empty robot scores 0; a robot with a non-finite coordinate or one beyond dead_bound is dead
 * and scores -infinity. */
double orc_robot_fitness(const orc_robot* R, const orc_params* p)
{
    if (R->M == 0) return 0.0;
    double sx = 0.0;
    for (int m = 0; m < R->M; ++m) {
        for (int q = 0; q < 3; ++q) {
            double c = R->x[3 * m + q];
            if (!isfinite(c) || fabs(c) > p->dead_bound) return -INFINITY;
        }
        sx += R->x[3 * m + 0];
    }
    return sx / R->M - R->x0_centroid;
}

/* ------------------------------------------------------------------------------------------ */
/* Population runner (OpenMP over robots only).                                                 */
/* ------------------------------------------------------------------------------------------ */

/* Build and simulate P robots (voxel grids concatenated, robot r at voxel_off[r]), write the
 * fitness and optionally the final positions (robot r's masses at mass_off[r], 3 doubles each),
 * and the mass / spring counts.  w, kappa, phi are per voxel or NULL.  nthreads <= 0 uses the
 * OpenMP default; a positive count holds for this call only.  Returns the number of threads used. */
int orc_run_population(int P, const int32_t* dims, const int64_t* voxel_off, const uint8_t* mats,
                       const double* w, const double* kappa, const double* phi,
                       const orc_params* p, int apply_lcc, int nsteps, int nthreads,
                       double* fitness_out, int32_t* M_out, int32_t* S_out,
                       const int64_t* mass_off, double* x_out)
{
    int used = 1;
#ifdef _OPENMP
    /* a num_threads clause, not omp_set_num_threads: a request applies to this call only */
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel num_threads(nt)
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int r = 0; r < P; ++r) {
        int64_t o = voxel_off[r];
        orc_robot* R = orc_robot_new(dims[3 * r], dims[3 * r + 1], dims[3 * r + 2], mats + o,
                                     w ? w + o : NULL, kappa ? kappa + o : NULL,
                                     phi ? phi + o : NULL, p, apply_lcc);
        orc_robot_simulate(R, p, nsteps);
        if (fitness_out) fitness_out[r] = orc_robot_fitness(R, p);
        if (M_out) M_out[r] = R->M;
        if (S_out) S_out[r] = R->S;
        if (x_out && mass_off) memcpy(x_out + 3 * mass_off[r], R->x, sizeof(double) * 3 * (size_t)R->M);
        orc_robot_free(R);
    }
    return used;
}

/* ------------------------------------------------------------------------------------------ */
/* Evolution generation (Section II-C; Table I): elite selection, uniform crossover, mutation.  */
/* ------------------------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014) used as a counter-based generator: output number `ctr` of the stream seeded
 * with `seed` is the SplitMix64 finaliser applied to seed + (ctr + 1) * 0x9E3779B97F4A7C15. */
static uint64_t orc_splitmix64(uint64_t seed, uint64_t ctr)
{
    uint64_t z = seed + (ctr + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Purposes of the random numbers of one generation. */
enum { ORC_RNG_PARENT_A = 0, ORC_RNG_PARENT_B = 1, ORC_RNG_MASK = 2, ORC_RNG_MUTATE = 3,
       ORC_RNG_GAUSS_U1 = 4, ORC_RNG_GAUSS_U2 = 5, ORC_RNG_CROSS = 6 };

/* Counter of the draw for (generation, child, gene, purpose): the fields are packed as
 * generation | child (16 bits) | gene (26 bits) | purpose (3 bits). */
static uint32_t orc_draw(uint64_t seed, uint64_t gen, uint64_t child, uint64_t gene, uint64_t purpose)
{
    uint64_t ctr = ((((gen << 16) | child) << 26 | gene) << 3) | purpose;
    return (uint32_t)(orc_splitmix64(seed, ctr) >> 32);
}

/* Exposed for the generator's statistical pins. */
uint32_t orc_rng_draw(uint64_t seed, uint64_t gen, uint64_t child, uint64_t gene, uint64_t purpose)
{
    return orc_draw(seed, gen, child, gene, purpose);
}

static const double* g_rank_key;  /* comparator context for the rank sort (single-threaded) */

static int cmp_rank(const void* p, const void* q)
{
    int a = *(const int*)p, b = *(const int*)q;
    double ka = g_rank_key[a], kb = g_rank_key[b];
    if (ka > kb) return -1;
    if (ka < kb) return 1;
    return (a > b) - (a < b);
}

/* One generation of the evolutionary step (Section II-C: elite selection, crossover and
 * mutation; Table I rates).
 * Rank: fitness descending, ties by ascending index, NaN counted as -infinity.
 * The E best genomes are copied unchanged into slots 0..E-1 in rank order.  Every slot c >= E
 * is a child of two elites: parent ranks floor(u * E / 2^32) for the draws (c, PARENT_A) and
 * (c, PARENT_B).  Uniform crossover: gene j comes from parent A when the top bit of draw
 * (c, j, MASK) is set, else from parent B; with a crossover rate below 1 (Table I: 0.4), a child
 * whose draw (c, CROSS) is below keep_threshold = floor((1 - rate) 2^32) takes every gene from
 * parent A instead (0 = always cross).  Mutation: when draw (c, j, MUTATE) < mut_threshold
 * the gene gets sigma * z added, z = sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller) with
 * u1 = (draw(c, j, U1) + 1) / 2^32 and u2 = draw(c, j, U2) / 2^32.
 * order_out[P] receives the rank order, parents_out[2P] the parent genome indices (elites name
 * themselves twice), mask_out / mutate_out[P*G] the per-gene crossover and mutation decisions
 * (0 for elites).  All outputs but genomes_out are optional.  Returns 0, or -1 on bad sizes. */
int orc_evo_generation(int P, int G, const double* fitness, const float* genomes_in,
                       double* genomes_out, int E, uint64_t seed, uint64_t gen,
                       uint32_t mut_threshold, double sigma, uint32_t keep_threshold,
                       int32_t* order_out, int32_t* parents_out, uint8_t* mask_out,
                       uint8_t* mutate_out)
{
    if (P <= 0 || G <= 0 || E <= 0 || E > P || P > 65536 || G > (1 << 26)) return -1;
    double* key = (double*)malloc(sizeof(double) * (size_t)P);
    int* order = (int*)malloc(sizeof(int) * (size_t)P);
    for (int i = 0; i < P; ++i) { key[i] = isnan(fitness[i]) ? -INFINITY : fitness[i]; order[i] = i; }
    g_rank_key = key;
    qsort(order, (size_t)P, sizeof(int), cmp_rank);
    for (int r = 0; r < E; ++r) {
        for (int j = 0; j < G; ++j) genomes_out[(size_t)r * G + j] = genomes_in[(size_t)order[r] * G + j];
        if (parents_out) { parents_out[2 * r] = order[r]; parents_out[2 * r + 1] = order[r]; }
        if (mask_out) memset(mask_out + (size_t)r * G, 0, (size_t)G);
        if (mutate_out) memset(mutate_out + (size_t)r * G, 0, (size_t)G);
    }
    for (int c = E; c < P; ++c) {
        uint32_t ua = orc_draw(seed, gen, (uint64_t)c, 0, ORC_RNG_PARENT_A);
        uint32_t ub = orc_draw(seed, gen, (uint64_t)c, 0, ORC_RNG_PARENT_B);
        int pa = order[(int)(((uint64_t)ua * (uint64_t)E) >> 32)];
        int pb = order[(int)(((uint64_t)ub * (uint64_t)E) >> 32)];
        if (parents_out) { parents_out[2 * c] = pa; parents_out[2 * c + 1] = pb; }
        int copy_a = orc_draw(seed, gen, (uint64_t)c, 0, ORC_RNG_CROSS) < keep_threshold;
        for (int j = 0; j < G; ++j) {
            int from_a = copy_a ? 1 : (int)(orc_draw(seed, gen, (uint64_t)c, (uint64_t)j, ORC_RNG_MASK) >> 31);
            double g = from_a ? genomes_in[(size_t)pa * G + j] : genomes_in[(size_t)pb * G + j];
            int mut = orc_draw(seed, gen, (uint64_t)c, (uint64_t)j, ORC_RNG_MUTATE) < mut_threshold;
            if (mut) {
                double u1 = ((double)orc_draw(seed, gen, (uint64_t)c, (uint64_t)j, ORC_RNG_GAUSS_U1) + 1.0) * 0x1p-32;
                double u2 = (double)orc_draw(seed, gen, (uint64_t)c, (uint64_t)j, ORC_RNG_GAUSS_U2) * 0x1p-32;
                double z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
                g = g + sigma * z;
            }
            genomes_out[(size_t)c * G + j] = g;
            if (mask_out) mask_out[(size_t)c * G + j] = (uint8_t)from_a;
            if (mutate_out) mutate_out[(size_t)c * G + j] = (uint8_t)mut;
        }
    }
    if (order_out) for (int i = 0; i < P; ++i) order_out[i] = order[i];
    free(key);
    free(order);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Adjoint (reverse mode) of the time stepping.                                                 */
/* ------------------------------------------------------------------------------------------ */

/* Fitness of a freshly built robot after nsteps, plus a hash of its contact-mode sequence, so a
 * finite-difference sample whose +h and -h runs took different contact modes can be discarded.
 * Parameters as for orc_robot_new. */
double orc_fitness_after_modes(int nx, int ny, int nz, const uint8_t* mat, const double* w,
                               const double* kappa, const double* phi, const orc_params* p,
                               int apply_lcc, int nsteps, const uint8_t* force, uint8_t* modes_out,
                               uint64_t* mode_hash);

double orc_fitness_after(int nx, int ny, int nz, const uint8_t* mat, const double* w,
                         const double* kappa, const double* phi, const orc_params* p,
                         int apply_lcc, int nsteps, uint64_t* mode_hash)
{
    return orc_fitness_after_modes(nx, ny, nz, mat, w, kappa, phi, p, apply_lcc, nsteps, NULL, NULL,
                                   mode_hash);
}

/* orc_fitness_after with the contact modes of every step recorded (modes_out, nsteps x M in mass
 * order, optional) or imposed (force, nsteps x M, optional; see orc_step). */
double orc_fitness_after_modes(int nx, int ny, int nz, const uint8_t* mat, const double* w,
                               const double* kappa, const double* phi, const orc_params* p,
                               int apply_lcc, int nsteps, const uint8_t* force, uint8_t* modes_out,
                               uint64_t* mode_hash)
{
    orc_robot* R = orc_robot_new(nx, ny, nz, mat, w, kappa, phi, p, apply_lcc);
    double* F = (double*)malloc(sizeof(double) * 3 * (size_t)(R->M > 0 ? R->M : 1));
    uint8_t* modes = (uint8_t*)malloc((size_t)(R->M > 0 ? R->M : 1));
    uint64_t h = 1469598103934665603ull;   /* FNV-1a over all modes of all steps */
    for (int n = 0; n < nsteps; ++n) {
        orc_step(R, p, F, modes, NULL, force ? force + (size_t)n * (size_t)R->M : NULL);
        if (modes_out) memcpy(modes_out + (size_t)n * (size_t)R->M, modes, (size_t)R->M);
        for (int m = 0; m < R->M; ++m) { h ^= modes[m]; h *= 1099511628211ull; }
    }
    double f = orc_robot_fitness(R, p);
    if (mode_hash) *mode_hash = h;
    free(F); free(modes);
    orc_robot_free(R);
    return f;
}

/* Gradient of L = dL_df * fitness after nsteps with respect to the per-voxel material weight w,
 * stiffness kappa and actuation phase phi, for a freshly built robot (parameters as for
 * orc_robot_new; w, kappa, phi may be NULL for the material defaults).
 * The voxel parametrisation: k_v = w_v kappa_v, a_v = w_v amp_mat[material_v], phase phi_v.
 * The forward run stores every state; the reverse sweep runs the exact transpose of each step
 * with the contact modes of the forward run held fixed (the mode switches are measure-zero
 * events where the map is not differentiable).  Gradients of empty voxels are 0.
 * lx_final (optional, 3M doubles) replaces the fitness term by a general terminal loss
 * L = sum_i lx_final_i . x_i(N).  Returns the fitness of the forward run. */
double orc_robot_adjoint(int nx, int ny, int nz, const uint8_t* mat, const double* w,
                         const double* kappa, const double* phi, const orc_params* p,
                         int apply_lcc, int nsteps, double dL_df, const double* lx_final,
                         double* g_w, double* g_kappa, double* g_phi)
{
    orc_robot* R = orc_robot_new(nx, ny, nz, mat, w, kappa, phi, p, apply_lcc);
    int M = R->M, S = R->S, V = R->V;
    size_t M3 = 3 * (size_t)(M > 0 ? M : 1);
    double* X = (double*)malloc(sizeof(double) * M3 * (size_t)(nsteps + 1));
    double* Fh = (double*)malloc(sizeof(double) * M3 * (size_t)(nsteps > 0 ? nsteps : 1));
    uint8_t* modes = (uint8_t*)malloc((size_t)(M > 0 ? M : 1) * (size_t)(nsteps > 0 ? nsteps : 1));
    double* F = (double*)malloc(sizeof(double) * M3);
    /* forward, keeping x_n, the pre-contact force and the contact modes of every step */
    for (int n = 0; n < nsteps; ++n) {
        memcpy(X + (size_t)n * M3, R->x, sizeof(double) * 3 * (size_t)M);
        orc_step(R, p, F, modes + (size_t)n * (size_t)M, Fh + (size_t)n * M3, NULL);
    }
    memcpy(X + (size_t)nsteps * M3, R->x, sizeof(double) * 3 * (size_t)M);
    double fit = orc_robot_fitness(R, p);

    double* lx = (double*)calloc(M3, sizeof(double));
    double* lv = (double*)calloc(M3, sizeof(double));
    double* lF = (double*)malloc(sizeof(double) * M3);
    size_t Sc = (size_t)(S > 0 ? S : 1);
    double* lk = (double*)calloc(Sc, sizeof(double));
    double* la = (double*)calloc(Sc, sizeof(double));
    double* lb = (double*)calloc(Sc, sizeof(double));
    if (lx_final) memcpy(lx, lx_final, sizeof(double) * 3 * (size_t)M);
    else for (int m = 0; m < M; ++m) lx[3 * m] = dL_df / M;   /* dL/dx_N of the centroid term */

    const double c = p->damping, dt = p->dt, mass = p->mass;
    for (int n = nsteps - 1; n >= 0; --n) {
        const double* xn = X + (size_t)n * M3;
        const double* Fp = Fh + (size_t)n * M3;
        const uint8_t* md = modes + (size_t)n * (size_t)M;
        /* integration and contact, per mass; lx keeps the direct x_{n+1} -> x_n term */
        for (int m = 0; m < M; ++m) {
            double lv1[3], lvt[3], lFt[3];
            for (int q = 0; q < 3; ++q) {
                lv1[q] = lv[3 * m + q] + dt * lx[3 * m + q];
                lvt[q] = c * lv1[q];
                lFt[q] = c * dt / mass * lv1[q];
            }
            if (md[m] == ORC_FREE) {
                for (int q = 0; q < 3; ++q) { lF[3 * m + q] = lFt[q]; lv[3 * m + q] = lvt[q]; }
            } else if (md[m] == ORC_STICK) {
                lF[3 * m + 0] = 0.0; lF[3 * m + 1] = 0.0; lF[3 * m + 2] = lFt[2];
                lv[3 * m + 0] = 0.0; lv[3 * m + 1] = 0.0; lv[3 * m + 2] = lvt[2];
                lx[3 * m + 2] += lFt[2] * (-p->k_ground);
            } else if (md[m] == ORC_SLIP_HELD) {
                /* F_h cancelled, velocity kept: only the normal force depends on the state */
                lF[3 * m + 0] = 0.0; lF[3 * m + 1] = 0.0; lF[3 * m + 2] = lFt[2];
                for (int q = 0; q < 3; ++q) lv[3 * m + q] = lvt[q];
                lx[3 * m + 2] += lFt[2] * (-p->k_ground);
            } else {
                double fn = p->k_ground * (-xn[3 * m + 2]);
                double fx = Fp[3 * m + 0], fy = Fp[3 * m + 1];
                double fh = sqrt(fx * fx + fy * fy);
                double ux = fx / fh, uy = fy / fh, r = p->mu_k * fn;
                double ul = ux * lFt[0] + uy * lFt[1];
                lF[3 * m + 0] = lFt[0] - (r / fh) * (lFt[0] - ux * ul);
                lF[3 * m + 1] = lFt[1] - (r / fh) * (lFt[1] - uy * ul);
                lF[3 * m + 2] = lFt[2];
                double lfn = -p->mu_k * ul + lFt[2];
                lx[3 * m + 2] += lfn * (-p->k_ground);
                for (int q = 0; q < 3; ++q) lv[3 * m + q] = lvt[q];
            }
        }
        /* springs: f = k (l - L) d / l added to a, subtracted from b */
        const double t = (double)n * p->dt;
        const double wt = 2.0 * M_PI * p->freq * t;
        const double sn = sin(wt), cs = cos(wt);
        for (int s = 0; s < S; ++s) {
            int a = R->sa[s], b = R->sb[s];
            double d[3], lf[3];
            for (int q = 0; q < 3; ++q) {
                d[q] = xn[3 * b + q] - xn[3 * a + q];
                lf[q] = lF[3 * a + q] - lF[3 * b + q];
            }
            double l = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (l < 1e-12) continue;
            double u[3] = {d[0] / l, d[1] / l, d[2] / l};
            double L = R->L0[s] * (1.0 + R->alpha[s] * sn + R->beta[s] * cs);
            double ulf = u[0] * lf[0] + u[1] * lf[1] + u[2] * lf[2];
            double k = R->ks[s];
            for (int q = 0; q < 3; ++q) {
                double ld = k * ((1.0 - L / l) * lf[q] + (L / l) * u[q] * ulf);
                lx[3 * b + q] += ld;
                lx[3 * a + q] -= ld;
            }
            lk[s] += (l - L) * ulf;
            double lL = -k * ulf;
            la[s] += lL * R->L0[s] * sn;
            lb[s] += lL * R->L0[s] * cs;
        }
    }
    /* per-spring sensitivities -> per-voxel parameters */
    double* lkv = (double*)calloc((size_t)(V > 0 ? V : 1), sizeof(double));
    double* lav = (double*)calloc((size_t)(V > 0 ? V : 1), sizeof(double));
    double* lbv = (double*)calloc((size_t)(V > 0 ? V : 1), sizeof(double));
    for (int s = 0; s < S; ++s) {
        int n = R->s_ninc[s];
        for (int t = 0; t < n; ++t) {
            int v = R->s_vox[4 * s + t];
            lkv[v] += lk[s] / n; lav[v] += la[s] / n; lbv[v] += lb[s] / n;
        }
    }
    for (int v = 0; v < V; ++v) {
        double A = p->amp_mat[R->mat[v]];
        double cp = cos(R->phi[v]), sp = sin(R->phi[v]);
        if (R->mat[v] == 0) {
            if (g_w) g_w[v] = 0.0;
            if (g_kappa) g_kappa[v] = 0.0;
            if (g_phi) g_phi[v] = 0.0;
            continue;
        }
        if (g_w) g_w[v] = R->kappa[v] * lkv[v] + A * (cp * lav[v] + sp * lbv[v]);
        if (g_kappa) g_kappa[v] = R->w[v] * lkv[v];
        if (g_phi) g_phi[v] = R->w[v] * A * (-sp * lav[v] + cp * lbv[v]);
    }
    free(lkv); free(lav); free(lbv);
    free(lx); free(lv); free(lF); free(lk); free(la); free(lb);
    free(X); free(Fh); free(modes); free(F);
    orc_robot_free(R);
    return fit;
}

/* ------------------------------------------------------------------------------------------ */
/* Population diversity (the paper's Fig. 3(b) "diversity curve"; definitions taken here).      */
/* ------------------------------------------------------------------------------------------ */

/* Root mean square of the pairwise Euclidean distances between P genomes of G values, summed
 * over all ordered pairs i != j (plain double loops). */
double orc_genome_diversity(int P, int G, const float* g)
{
    double acc = 0.0;
    for (int i = 0; i < P; ++i)
        for (int j = 0; j < P; ++j) {
            if (i == j) continue;
            double d2 = 0.0;
            for (int k = 0; k < G; ++k) {
                double d = (double)g[(size_t)i * G + k] - (double)g[(size_t)j * G + k];
                d2 += d * d;
            }
            acc += d2;
        }
    return sqrt(acc / ((double)P * (P - 1)));
}

/* Mean over unordered robot pairs of the fraction of voxels (V per robot) whose materials
 * differ. */
double orc_morphology_diversity(int P, int V, const uint8_t* mat)
{
    double acc = 0.0;
    for (int i = 0; i < P; ++i)
        for (int j = i + 1; j < P; ++j) {
            int diff = 0;
            for (int v = 0; v < V; ++v) diff += mat[(size_t)i * V + v] != mat[(size_t)j * V + v];
            acc += (double)diff / V;
        }
    return acc / (0.5 * P * (P - 1));
}
