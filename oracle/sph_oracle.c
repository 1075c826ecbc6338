/*
 * sph_oracle.c -- plain, slow FP64 CPU oracle for the SPH view path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load this
 * library.  The CUDA library never includes, links or calls anything here, and this file includes nothing of
 * the CUDA side: the two share no code, no headers and no constants.
 *
 * What it computes, and where each piece comes from:
 *   - the view operators of the paper's Section 4 (Eq. 3-5): narrowing+AoS->SoA gather of the read set A_in
 *     (the "prologue" of Section 3.1) and the widening SoA->AoS scatter of the write set A_out (the
 *     "epilogue");  or_gather_f64 / or_gather_f32 / or_gather_pos_f32 / or_scatter_f64 / or_scatter_f32;
 *   - the cell bucketing of Section 2.1 (cells at least as wide as the interaction radius; particles of one
 *     cell stored as one contiguous chunk as in Section 2.2 and the chunk lists of Section 5.2):  or_bin;
 *   - the density and force sums of Section 2.1 (steps 1 and 2) written as their plain definitions: a sum over
 *     ALL particle pairs with the predicate of Listing 1 as a branch (no cell list, no masking), in the periodic
 *     minimum image.  The paper fixes no SPH formula; the textbook forms used are the 3D cubic spline
 *     (Monaghan & Lattanzio 1985), an ideal-gas EOS and the Monaghan (1992) artificial viscosity, with the
 *     symmetrised momentum / energy equations of Price (2012);  or_density / or_eos / or_force;
 *   - the FP64 global momentum and energy sums; or_reduce.
 *   - the leapfrog kick-drift-kick of Section 2.1 (steps 3-5); or_kick / or_drift, and or_drift_walls for
 *     open boxes (reflecting walls).
 *   - the smoothing-length iteration of Section 2.1 step 1 (density, grow or shrink h, repeat until every
 *     particle meets its termination test); or_h_iterate.
 *   - the paper's own kernel, the quartic spline M5 (Section 2.1), next to the cubic spline; and the fuller
 *     density and force views its Section 2.1 and Table 1 describe (neighbour count, velocity divergence and
 *     rotation, the smoothing-length derivative terms): or_kw / or_kdwdr / or_kdwdh, or_density_ext,
 *     or_force_ext.  The paper prints none of these formulas; the textbook forms used are named there.
 *
 * Compile with -ffp-contract=off: every product and sum below is rounded on its own, exactly as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* ---------------------------------------------------------------------------------------------------------
 * Kernel: 3D cubic spline with support 2h (Monaghan & Lattanzio 1985).  W(r,h) = f(q) / (pi h^3), q = r/h,
 *   f(q) = 1 - 3/2 q^2 + 3/4 q^3   (0 <= q < 1)
 *        = 1/4 (2 - q)^3           (1 <= q < 2)
 *        = 0                        (q >= 2)
 * dW/dr = f'(q) / (pi h^4), f'(q) = -3 q + 9/4 q^2 (q < 1), -3/4 (2 - q)^2 (1 <= q < 2), 0 otherwise.
 * ------------------------------------------------------------------------------------------------------- */
double or_w(double r, double h)
{
    double q = r / h;
    double f;
    if (q < 1.0) {
        f = 1.0 - 1.5 * q * q + 0.75 * q * q * q;
    } else if (q < 2.0) {
        double t = 2.0 - q;
        f = 0.25 * t * t * t;
    } else {
        f = 0.0;
    }
    return f / (OR_PI * h * h * h);
}

double or_dwdr(double r, double h)
{
    double q = r / h;
    double fp;
    if (q < 1.0) {
        fp = -3.0 * q + 2.25 * q * q;
    } else if (q < 2.0) {
        double t = 2.0 - q;
        fp = -0.75 * t * t;
    } else {
        fp = 0.0;
    }
    return fp / (OR_PI * h * h * h * h);
}

void or_w_array(int64_t n, const double *r, const double *h, double *w)
{
    for (int64_t k = 0; k < n; ++k) w[k] = or_w(r[k], h[k]);
}

void or_dwdr_array(int64_t n, const double *r, const double *h, double *dw)
{
    for (int64_t k = 0; k < n; ++k) dw[k] = or_dwdr(r[k], h[k]);
}

/* Periodic minimum image of one coordinate difference (box edge L). */
static double or_min_image(double d, double L, int periodic)
{
    if (!periodic) return d;
    if (d > 0.5 * L) {
        d = d - L;
    } else if (d < -0.5 * L) {
        d = d + L;
    }
    return d;
}

/* ---------------------------------------------------------------------------------------------------------
 * Density (Section 2.1 step 1; Listing 1's DensityPredicate + Density as a branch):
 *   rho_i = sum_j m_j W(|r_ij|, h_i) over all j with |r_ij| < 2 h_i, the self term j = i included.
 * x is n x 3 (row = particle), targets lists the i to evaluate (nt of them), rho_out has nt entries.
 * ------------------------------------------------------------------------------------------------------- */
void or_density(int64_t n, const double *x, const double *m, const double *h, const double *box, int periodic,
                int64_t nt, const int64_t *targets, double *rho_out)
{
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets[t];
        double sum = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double dx = or_min_image(x[3 * i + 0] - x[3 * j + 0], box[0], periodic);
            double dy = or_min_image(x[3 * i + 1] - x[3 * j + 1], box[1], periodic);
            double dz = or_min_image(x[3 * i + 2] - x[3 * j + 2], box[2], periodic);
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (r < 2.0 * h[i]) {
                sum += m[j] * or_w(r, h[i]);
            }
        }
        rho_out[t] = sum;
    }
}

/* Ideal-gas equation of state: P = (gamma - 1) rho u, c_s = sqrt(gamma P / rho). */
void or_eos(int64_t n, const double *rho, const double *u, double gamma, double *P, double *cs)
{
    for (int64_t i = 0; i < n; ++i) {
        P[i] = (gamma - 1.0) * rho[i] * u[i];
        cs[i] = sqrt(gamma * P[i] / rho[i]);
    }
}

/* ---------------------------------------------------------------------------------------------------------
 * Force (Section 2.1 step 2), symmetrised SPH momentum and energy equations with Monaghan viscosity:
 *   a_i      = - sum_j m_j [ P_i/rho_i^2 grad_i W(r_ij,h_i) + P_j/rho_j^2 grad_i W(r_ij,h_j) + Pi_ij gradbar ]
 *   du_i/dt  =   sum_j m_j [ P_i/rho_i^2 v_ij . grad_i W(r_ij,h_i) + 1/2 Pi_ij v_ij . gradbar ]
 *   grad_i W(r_ij, h) = dW/dr(r, h) r_ij / r,  gradbar = (grad_i W(r_ij,h_i) + grad_i W(r_ij,h_j)) / 2,
 *   Pi_ij = (-alpha cbar mu + beta mu^2) / rhobar  if v_ij . r_ij < 0, else 0,
 *   mu = hbar v_ij . r_ij / (r^2 + eps hbar^2); hbar, cbar, rhobar are pair means.
 * Pairs: every j != i with |r_ij| < 2 max(h_i, h_j) (the force predicate; no symmetry is exploited, as in the
 * paper's Section 5.3).  A coincident pair (r = 0) contributes nothing: every term carries r_ij or v_ij . r_ij.
 * rho, P, cs must be valid for every j that lies within the support of a target.
 * ------------------------------------------------------------------------------------------------------- */
void or_force(int64_t n, const double *x, const double *v, const double *m, const double *h, const double *rho,
              const double *P, const double *cs, const double *box, int periodic, double alpha, double beta,
              double eps, int64_t nt, const int64_t *targets, double *a_out, double *dudt_out)
{
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets[t];
        double ax = 0.0, ay = 0.0, az = 0.0, du = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = or_min_image(x[3 * i + 0] - x[3 * j + 0], box[0], periodic);
            double dy = or_min_image(x[3 * i + 1] - x[3 * j + 1], box[1], periodic);
            double dz = or_min_image(x[3 * i + 2] - x[3 * j + 2], box[2], periodic);
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double hmax = h[i] > h[j] ? h[i] : h[j];
            if (!(r < 2.0 * hmax)) continue;
            if (r == 0.0) continue;
            double gi = or_dwdr(r, h[i]) / r; /* grad_i W(r_ij, h_i) = gi * r_ij */
            double gj = or_dwdr(r, h[j]) / r; /* grad_i W(r_ij, h_j) = gj * r_ij */
            double gbar = 0.5 * (gi + gj);
            double vx = v[3 * i + 0] - v[3 * j + 0];
            double vy = v[3 * i + 1] - v[3 * j + 1];
            double vz = v[3 * i + 2] - v[3 * j + 2];
            double vdotr = vx * dx + vy * dy + vz * dz;
            double visc = 0.0;
            if (vdotr < 0.0) {
                double hbar = 0.5 * (h[i] + h[j]);
                double mu = hbar * vdotr / (r * r + eps * hbar * hbar);
                double cbar = 0.5 * (cs[i] + cs[j]);
                double rhobar = 0.5 * (rho[i] + rho[j]);
                visc = (-alpha * cbar * mu + beta * mu * mu) / rhobar;
            }
            double Ai = P[i] / (rho[i] * rho[i]);
            double Aj = P[j] / (rho[j] * rho[j]);
            double coef = m[j] * (Ai * gi + Aj * gj + visc * gbar);
            ax -= coef * dx;
            ay -= coef * dy;
            az -= coef * dz;
            du += m[j] * (Ai * gi * vdotr + 0.5 * visc * gbar * vdotr);
        }
        a_out[3 * t + 0] = ax;
        a_out[3 * t + 1] = ay;
        a_out[3 * t + 2] = az;
        dudt_out[t] = du;
    }
}

/* Indices of all j within distance < rad_factor * max(h_i, h_j) of i (minimum image), j != i excluded iff
 * exclude_self.  Returns the count written (at most cap). Used to find the particles whose density a sampled
 * force evaluation depends on. */
int64_t or_neighbours(int64_t n, const double *x, const double *h, const double *box, int periodic, int64_t i,
                      double rad_factor, int64_t cap, int64_t *out)
{
    int64_t cnt = 0;
    for (int64_t j = 0; j < n; ++j) {
        double dx = or_min_image(x[3 * i + 0] - x[3 * j + 0], box[0], periodic);
        double dy = or_min_image(x[3 * i + 1] - x[3 * j + 1], box[1], periodic);
        double dz = or_min_image(x[3 * i + 2] - x[3 * j + 2], box[2], periodic);
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        double hmax = h[i] > h[j] ? h[i] : h[j];
        if (r < rad_factor * hmax) {
            if (cnt < cap) out[cnt] = j;
            ++cnt;
        }
    }
    return cnt;
}

/* ---------------------------------------------------------------------------------------------------------
 * Cell bucketing (Section 2.1: cells at least as wide as the interaction radius, particles sorted into them;
 * Section 2.2 / 5.2: the particles of one cell form one contiguous chunk, indexed by a CSR-like list).
 * Cell of a coordinate: k = floor(x * (ncell / box)), clamped into [0, ncell-1].  Linear cell index
 * c = kx + nx (ky + ny kz).  Slot order: cell-major, and inside a cell ascending particle index (a stable
 * counting sort).  Outputs: cell_of[i] per particle, cell_start[c] (ncells+1 entries), perm[s] = particle held
 * by slot s, cell_of_slot[s].  Returns the number of coordinates that fell outside [0, box] (they are clamped).
 * ------------------------------------------------------------------------------------------------------- */
int64_t or_bin(int64_t n, const double *x, const double *box, const int32_t *ncell, int32_t *cell_of,
               int32_t *cell_start, int32_t *perm, int32_t *cell_of_slot)
{
    int64_t bad = 0;
    int64_t ncells = (int64_t)ncell[0] * ncell[1] * ncell[2];
    for (int64_t i = 0; i < n; ++i) {
        int32_t k[3];
        for (int d = 0; d < 3; ++d) {
            double inv = (double)ncell[d] / box[d];
            double xv = x[3 * i + d];
            if (!(xv >= 0.0 && xv <= box[d])) ++bad;
            double f = floor(xv * inv);
            int32_t kk;
            if (!(f >= 0.0)) kk = 0;                       /* also catches NaN */
            else if (f > (double)(ncell[d] - 1)) kk = ncell[d] - 1;
            else kk = (int32_t)f;
            k[d] = kk;
        }
        cell_of[i] = k[0] + ncell[0] * (k[1] + ncell[1] * k[2]);
    }
    for (int64_t c = 0; c <= ncells; ++c) cell_start[c] = 0;
    for (int64_t i = 0; i < n; ++i) cell_start[cell_of[i] + 1] += 1;
    for (int64_t c = 0; c < ncells; ++c) cell_start[c + 1] += cell_start[c];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncells > 0 ? ncells : 1));
    for (int64_t c = 0; c < ncells; ++c) fill[c] = cell_start[c];
    for (int64_t i = 0; i < n; ++i) {
        int32_t s = fill[cell_of[i]]++;
        perm[s] = (int32_t)i;
        cell_of_slot[s] = cell_of[i];
    }
    free(fill);
    return bad;
}

/* ---------------------------------------------------------------------------------------------------------
 * Cell bucketing of independent patches (open boxes of edge box[d], patch p = particles patch_start[p] ..
 * patch_start[p+1]-1, patch-local positions).  Each patch gets its own grid, chosen so that every cell is at
 * least as wide as the largest interaction radius 2 h_max of the patch (Section 2.1): per axis
 * n = floor(box / (2 h_max)), at least 1, at most ncap, lowered while box / n < 2 h_max; n = ncap for a patch
 * without particles.  Global cell ids: patch_cell_base[p] + kx + nx (ky + ny kz) with k = floor(x * (n / box))
 * clamped into [0, n-1].  Slot order as in or_bin: cell-major, ascending particle index inside a cell.
 * Outputs patch_n (3 per patch), patch_cell_base (npatch + 1), cell_of, cell_start (cells + 1), perm,
 * cell_of_slot; returns the number of cells.
 * ------------------------------------------------------------------------------------------------------- */
int64_t or_bin_patches(int64_t n, const double *x, const double *h, const int64_t *patch_start, int32_t npatch,
                       const double *box, int32_t ncap, int32_t *patch_n, int32_t *patch_cell_base, int32_t *cell_of,
                       int32_t *cell_start, int32_t *perm, int32_t *cell_of_slot)
{
    patch_cell_base[0] = 0;
    for (int32_t p = 0; p < npatch; ++p) {
        double hm = 0.0;
        for (int64_t i = patch_start[p]; i < patch_start[p + 1]; ++i)
            if (h[i] > hm) hm = h[i];
        int32_t cells = 1;
        for (int d = 0; d < 3; ++d) {
            int32_t nn = ncap;
            if (hm > 0.0) {
                double f = floor(box[d] / (2.0 * hm));
                nn = f >= (double)ncap ? ncap : (f >= 1.0 ? (int32_t)f : 1);
                while (nn > 1 && box[d] / (double)nn < 2.0 * hm) --nn;
            }
            patch_n[3 * p + d] = nn;
            cells *= nn;
        }
        patch_cell_base[p + 1] = patch_cell_base[p] + cells;
    }
    int64_t ncells = patch_cell_base[npatch];
    for (int32_t p = 0; p < npatch; ++p) {
        for (int64_t i = patch_start[p]; i < patch_start[p + 1]; ++i) {
            int32_t k[3];
            for (int d = 0; d < 3; ++d) {
                int32_t nn = patch_n[3 * p + d];
                double inv = (double)nn / box[d];
                double f = floor(x[3 * i + d] * inv);
                k[d] = !(f >= 0.0) ? 0 : (f > (double)(nn - 1) ? nn - 1 : (int32_t)f);
            }
            cell_of[i] = patch_cell_base[p] + k[0] + patch_n[3 * p] * (k[1] + patch_n[3 * p + 1] * k[2]);
        }
    }
    for (int64_t c = 0; c <= ncells; ++c) cell_start[c] = 0;
    for (int64_t i = 0; i < n; ++i) cell_start[cell_of[i] + 1] += 1;
    for (int64_t c = 0; c < ncells; ++c) cell_start[c + 1] += cell_start[c];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncells > 0 ? ncells : 1));
    for (int64_t c = 0; c < ncells; ++c) fill[c] = cell_start[c];
    for (int64_t i = 0; i < n; ++i) {
        int32_t s = fill[cell_of[i]]++;
        perm[s] = (int32_t)i;
        cell_of_slot[s] = cell_of[i];
    }
    free(fill);
    return ncells;
}

/* FP32 patch-local positions relative to the origin of the slot's cell: (float)(x - k_d * (box_d / n_d)). */
void or_gather_pos_f32_patches(const uint8_t *aos, int64_t stride, int64_t n, const int32_t *perm, int64_t off,
                               const int32_t *cell_of_slot, const int32_t *patch_cell_base, const int32_t *patch_n,
                               int32_t npatch, const double *box, float *out)
{
    for (int64_t s = 0; s < n; ++s) {
        int32_t c = cell_of_slot[s];
        int32_t p = 0;
        while (p + 1 < npatch && patch_cell_base[p + 1] <= c) ++p;
        int32_t local = c - patch_cell_base[p];
        const int32_t *nn = patch_n + 3 * p;
        int32_t k[3] = {local % nn[0], (local / nn[0]) % nn[1], local / (nn[0] * nn[1])};
        for (int d = 0; d < 3; ++d) {
            double xv;
            memcpy(&xv, aos + (int64_t)perm[s] * stride + off + 8 * d, 8);
            double edge = box[d] / (double)nn[d];
            double origin = (double)k[d] * edge;
            out[(int64_t)d * n + s] = (float)(xv - origin);
        }
    }
}

/* ---------------------------------------------------------------------------------------------------------
 * View conversions (Section 4, Eq. 3-5).  The gather is narrowing N followed by C_AoS^SoA, fused: for every
 * slot s, out[comp][s] = field component of record perm[s].  The scatter is C_SoA^AoS followed by widening W:
 * the field of record perm[s] is overwritten from in[comp][s]; no other byte of the record is touched.
 * A field is ncomp contiguous doubles at byte offset off inside a record of `stride` bytes.  SoA storage is
 * component-major: component k of slot s lives at out[k * n + s].
 * ------------------------------------------------------------------------------------------------------- */
void or_gather_f64(const uint8_t *aos, int64_t stride, int64_t n, const int32_t *perm, int64_t off, int ncomp,
                   double *out)
{
    for (int k = 0; k < ncomp; ++k) {
        for (int64_t s = 0; s < n; ++s) {
            memcpy(&out[(int64_t)k * n + s], aos + (int64_t)perm[s] * stride + off + 8 * k, 8);
        }
    }
}

/* FP32 views: every value is the round-to-nearest cast of the double. */
void or_gather_f32(const uint8_t *aos, int64_t stride, int64_t n, const int32_t *perm, int64_t off, int ncomp,
                   float *out)
{
    for (int k = 0; k < ncomp; ++k) {
        for (int64_t s = 0; s < n; ++s) {
            double d;
            memcpy(&d, aos + (int64_t)perm[s] * stride + off + 8 * k, 8);
            out[(int64_t)k * n + s] = (float)d;
        }
    }
}

/* FP32 positions are stored relative to the origin of the slot's cell: (float)(x - k_d * (box_d / ncell_d)),
 * the subtraction and the product each rounded in FP64, then one round-to-nearest cast. */
void or_gather_pos_f32(const uint8_t *aos, int64_t stride, int64_t n, const int32_t *perm, int64_t off,
                       const int32_t *cell_of_slot, const double *box, const int32_t *ncell, float *out)
{
    for (int64_t s = 0; s < n; ++s) {
        int32_t c = cell_of_slot[s];
        int32_t k[3];
        k[0] = c % ncell[0];
        k[1] = (c / ncell[0]) % ncell[1];
        k[2] = c / (ncell[0] * ncell[1]);
        for (int d = 0; d < 3; ++d) {
            double xv;
            memcpy(&xv, aos + (int64_t)perm[s] * stride + off + 8 * d, 8);
            double edge = box[d] / (double)ncell[d];
            double origin = (double)k[d] * edge;
            out[(int64_t)d * n + s] = (float)(xv - origin);
        }
    }
}

void or_scatter_f64(uint8_t *aos, int64_t stride, int64_t n, const int32_t *perm, int64_t off, int ncomp,
                    const double *in)
{
    for (int k = 0; k < ncomp; ++k) {
        for (int64_t s = 0; s < n; ++s) {
            memcpy(aos + (int64_t)perm[s] * stride + off + 8 * k, &in[(int64_t)k * n + s], 8);
        }
    }
}

/* FP32 views widen exactly: (double)float. */
void or_scatter_f32(uint8_t *aos, int64_t stride, int64_t n, const int32_t *perm, int64_t off, int ncomp,
                    const float *in)
{
    for (int k = 0; k < ncomp; ++k) {
        for (int64_t s = 0; s < n; ++s) {
            double d = (double)in[(int64_t)k * n + s];
            memcpy(aos + (int64_t)perm[s] * stride + off + 8 * k, &d, 8);
        }
    }
}

/* FP32 cell-relative positions widen back to the box: k_d * (box_d / ncell_d) + (double)rel, each op rounded in
 * FP64. */
void or_scatter_pos_f32(uint8_t *aos, int64_t stride, int64_t n, const int32_t *perm, int64_t off,
                        const int32_t *cell_of_slot, const double *box, const int32_t *ncell, const float *in)
{
    for (int64_t s = 0; s < n; ++s) {
        int32_t c = cell_of_slot[s];
        int32_t k[3];
        k[0] = c % ncell[0];
        k[1] = (c / ncell[0]) % ncell[1];
        k[2] = c / (ncell[0] * ncell[1]);
        for (int d = 0; d < 3; ++d) {
            double edge = box[d] / (double)ncell[d];
            double xv = (double)k[d] * edge + (double)in[(int64_t)d * n + s];
            memcpy(aos + (int64_t)perm[s] * stride + off + 8 * d, &xv, 8);
        }
    }
}

/* ---------------------------------------------------------------------------------------------------------
 * FP64 global sums: out[0..2] = sum m v, out[3..5] = sum m a, out[6] = sum m (|v|^2/2 + u),
 * out[7] = sum m (v . a + du/dt).  Straight loop in particle order.
 * ------------------------------------------------------------------------------------------------------- */
void or_reduce(int64_t n, const double *m, const double *v, const double *a, const double *u,
               const double *dudt, double *out)
{
    for (int k = 0; k < 8; ++k) out[k] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        out[0] += m[i] * v[3 * i + 0];
        out[1] += m[i] * v[3 * i + 1];
        out[2] += m[i] * v[3 * i + 2];
        out[3] += m[i] * a[3 * i + 0];
        out[4] += m[i] * a[3 * i + 1];
        out[5] += m[i] * a[3 * i + 2];
        double v2 = v[3 * i + 0] * v[3 * i + 0] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2];
        out[6] += m[i] * (0.5 * v2 + u[i]);
        double va = v[3 * i + 0] * a[3 * i + 0] + v[3 * i + 1] * a[3 * i + 1] + v[3 * i + 2] * a[3 * i + 2];
        out[7] += m[i] * (va + dudt[i]);
    }
}

/* ---------------------------------------------------------------------------------------------------------
 * Leapfrog pieces (Section 2.1 steps 3-5): a kick v += a dt_k, u += du/dt dt_k, and a drift x += v dt followed
 * by the periodic wrap into [0, box) (x - box if x >= box, x + box if x < 0).
 * ------------------------------------------------------------------------------------------------------- */
void or_kick(int64_t n, double dtk, const double *a, const double *dudt, double *v, double *u)
{
    for (int64_t i = 0; i < n; ++i) {
        v[3 * i + 0] = v[3 * i + 0] + a[3 * i + 0] * dtk;
        v[3 * i + 1] = v[3 * i + 1] + a[3 * i + 1] * dtk;
        v[3 * i + 2] = v[3 * i + 2] + a[3 * i + 2] * dtk;
        u[i] = u[i] + dudt[i] * dtk;
    }
}

void or_drift(int64_t n, double dt, const double *v, const double *box, int periodic, double *x)
{
    for (int64_t i = 0; i < n; ++i) {
        for (int d = 0; d < 3; ++d) {
            double xn = x[3 * i + d] + v[3 * i + d] * dt;
            if (periodic) {
                if (xn >= box[d]) xn = xn - box[d];
                else if (xn < 0.0) xn = xn + box[d];
            }
            x[3 * i + d] = xn;
        }
    }
}

/* ---------------------------------------------------------------------------------------------------------
 * Drift in an open box [0, box] with reflecting walls (the walls of an isolated patch; the paper's periodic
 * and ghost-cell boundaries do not apply to a patch that shares no particles with any other).  Per axis:
 * xn = x + v dt; a position past a wall is mirrored back through it and that velocity component changes sign
 * (xn < 0: xn = -xn; xn > box: xn = 2 box - xn); a position still outside after one mirror (|v dt| > box) is
 * clamped onto the wall.  x and v are updated in place.
 * ------------------------------------------------------------------------------------------------------- */
void or_drift_walls(int64_t n, double dt, double *v, const double *box, double *x)
{
    for (int64_t i = 0; i < n; ++i) {
        for (int d = 0; d < 3; ++d) {
            double xn = x[3 * i + d] + v[3 * i + d] * dt;
            if (xn < 0.0) {
                xn = -xn;
                v[3 * i + d] = -v[3 * i + d];
            } else if (xn > box[d]) {
                xn = (box[d] + box[d]) - xn;
                v[3 * i + d] = -v[3 * i + d];
            }
            if (xn < 0.0) xn = 0.0;
            else if (xn > box[d]) xn = box[d];
            x[3 * i + d] = xn;
        }
    }
}

/* ---------------------------------------------------------------------------------------------------------
 * Smoothing-length iteration (Section 2.1, step 1: compute the density, decide to grow or shrink the
 * interaction radius, recompute, until every particle meets its termination criterion).  The paper gives no
 * update rule; the one used is h <- eta (m_i / rho_i)^(1/3), which at uniform density rho = m / s^3 gives
 * h = eta s, with the termination test |h_new - h| < tol h, in FP64.  A particle that passes is frozen at
 * h_new.  Every round recomputes the densities of the particles not yet frozen (rho_i depends on h_i only);
 * after the last round the densities of all particles are recomputed at their final h.
 * h is updated in place; rho_out receives the final densities; *iters_out the number of rounds run (at most
 * max_iter).  Returns the number of particles still not frozen after the last round (0 = converged).
 * ------------------------------------------------------------------------------------------------------- */
int64_t or_h_iterate(int64_t n, const double *x, const double *m, double *h, const double *box, int periodic,
                     double eta, double tol, int32_t max_iter, double *rho_out, int32_t *iters_out)
{
    unsigned char *done = (unsigned char *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t *targets = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    double *rho_t = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *h_new = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int64_t undone = n;
    int32_t it = 0;
    while (undone > 0 && it < max_iter) {
        ++it;
        int64_t nt = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (!done[i]) targets[nt++] = i;
        }
        or_density(n, x, m, h, box, periodic, nt, targets, rho_t);
        for (int64_t t = 0; t < nt; ++t) {
            int64_t i = targets[t];
            h_new[t] = eta * cbrt(m[i] / rho_t[t]);
            if (fabs(h_new[t] - h[i]) < tol * h[i]) done[i] = 1;
        }
        for (int64_t t = 0; t < nt; ++t) h[targets[t]] = h_new[t];
        undone = 0;
        for (int64_t i = 0; i < n; ++i) undone += done[i] ? 0 : 1;
    }
    for (int64_t i = 0; i < n; ++i) targets[i] = i;
    or_density(n, x, m, h, box, periodic, n, targets, rho_out);
    *iters_out = it;
    free(done);
    free(targets);
    free(rho_t);
    free(h_new);
    return undone;
}

/* ---------------------------------------------------------------------------------------------------------
 * Kernel families (3D).  W(r, h) = sigma f(q) / h^3 with q = r / h and support q < kappa, written as sums of
 * truncated powers (t)_+ = max(t, 0):
 *   kern 0, cubic spline M4 (Monaghan & Lattanzio 1985): kappa = 2, sigma = 1/pi,
 *     f(q) = 1/4 (2 - q)_+^3 - (1 - q)_+^3          (= 1 - 3/2 q^2 + 3/4 q^3 for q < 1, 1/4 (2 - q)^3 for q < 2);
 *   kern 1, quartic spline M5 (Monaghan 1985; the paper's kernel, Section 2.1): kappa = 5/2, sigma = 1/(20 pi),
 *     f(q) = (5/2 - q)_+^4 - 5 (3/2 - q)_+^4 + 10 (1/2 - q)_+^4.
 * Derivatives: dW/dr = sigma f'(q) / h^4, and dW/dh = -sigma (3 f(q) + q f'(q)) / h^4 (d/dh of h^-3 f(r/h)).
 * ------------------------------------------------------------------------------------------------------- */
static double or_pos(double t) { return t > 0.0 ? t : 0.0; }

double or_kappa(int kern) { return kern == 1 ? 2.5 : 2.0; }

static double or_ksigma(int kern) { return kern == 1 ? 1.0 / (20.0 * OR_PI) : 1.0 / OR_PI; }

static double or_kf(int kern, double q)
{
    if (kern == 1) {
        double a = or_pos(2.5 - q), b = or_pos(1.5 - q), c = or_pos(0.5 - q);
        return a * a * a * a - 5.0 * (b * b * b * b) + 10.0 * (c * c * c * c);
    }
    double a = or_pos(2.0 - q), b = or_pos(1.0 - q);
    return 0.25 * (a * a * a) - b * b * b;
}

static double or_kfp(int kern, double q)
{
    if (kern == 1) {
        double a = or_pos(2.5 - q), b = or_pos(1.5 - q), c = or_pos(0.5 - q);
        return -4.0 * (a * a * a) + 20.0 * (b * b * b) - 40.0 * (c * c * c);
    }
    double a = or_pos(2.0 - q), b = or_pos(1.0 - q);
    return -0.75 * (a * a) + 3.0 * (b * b);
}

double or_kw(int kern, double r, double h)
{
    double q = r / h;
    return or_ksigma(kern) * or_kf(kern, q) / (h * h * h);
}

double or_kdwdr(int kern, double r, double h)
{
    double q = r / h;
    return or_ksigma(kern) * or_kfp(kern, q) / (h * h * h * h);
}

double or_kdwdh(int kern, double r, double h)
{
    double q = r / h;
    return -or_ksigma(kern) * (3.0 * or_kf(kern, q) + q * or_kfp(kern, q)) / (h * h * h * h);
}

/* which: 0 W, 1 dW/dr, 2 dW/dh, elementwise */
void or_kernel_array(int kern, int which, int64_t n, const double *r, const double *h, double *out)
{
    for (int64_t k = 0; k < n; ++k) {
        if (which == 0) out[k] = or_kw(kern, r[k], h[k]);
        else if (which == 1) out[k] = or_kdwdr(kern, r[k], h[k]);
        else out[k] = or_kdwdh(kern, r[k], h[k]);
    }
}

/* ---------------------------------------------------------------------------------------------------------
 * The fuller density view (Section 2.1 step 1 "the neighbour count, the rotational velocity vector, and
 * various derivative properties"; Table 1's larger density sets).  For each target i, over every j with
 * |r_ij| < kappa h_i (self included where it contributes):
 *   rho_i         = sum_j m_j W(r_ij, h_i)
 *   drho_i/dh_i   = sum_j m_j dW/dh(r_ij, h_i)
 *   Omega_i       = 1 + h_i / (3 rho_i) drho_i/dh_i   (the grad-h term of Springel & Hernquist 2002 / Price 2012
 *                                                       in 3D, where h ~ rho^(-1/3))
 *   n_i           = number of j != i with |r_ij| < kappa h_i
 *   (div v)_i     = -1/rho_i sum_j m_j v_ij . grad_i W(r_ij, h_i)
 *   (curl v)_i    =  1/rho_i sum_j m_j v_ij x grad_i W(r_ij, h_i)
 * with v_ij = v_i - v_j and grad_i W(r_ij, h) = dW/dr(r, h) r_ij / r (no contribution at r = 0).  On a uniform
 * lattice the two velocity estimates return 3c for v = c x and 2 w for v = w x x.  curl_out is nt x 3.
 * ------------------------------------------------------------------------------------------------------- */
void or_density_ext(int kern, int64_t n, const double *x, const double *v, const double *m, const double *h,
                    const double *box, int periodic, int64_t nt, const int64_t *targets, double *rho_out,
                    double *omega_out, double *nnb_out, double *divv_out, double *curl_out)
{
    double kap = or_kappa(kern);
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets[t];
        double rho = 0.0, drho = 0.0, cnt = 0.0, dv = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double dx = or_min_image(x[3 * i + 0] - x[3 * j + 0], box[0], periodic);
            double dy = or_min_image(x[3 * i + 1] - x[3 * j + 1], box[1], periodic);
            double dz = or_min_image(x[3 * i + 2] - x[3 * j + 2], box[2], periodic);
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (!(r < kap * h[i])) continue;
            rho += m[j] * or_kw(kern, r, h[i]);
            drho += m[j] * or_kdwdh(kern, r, h[i]);
            if (j != i) cnt += 1.0;
            if (r > 0.0) {
                double g = or_kdwdr(kern, r, h[i]) / r; /* grad_i W = g r_ij */
                double vx = v[3 * i + 0] - v[3 * j + 0];
                double vy = v[3 * i + 1] - v[3 * j + 1];
                double vz = v[3 * i + 2] - v[3 * j + 2];
                dv += m[j] * g * (vx * dx + vy * dy + vz * dz);
                cx += m[j] * g * (vy * dz - vz * dy);
                cy += m[j] * g * (vz * dx - vx * dz);
                cz += m[j] * g * (vx * dy - vy * dx);
            }
        }
        rho_out[t] = rho;
        omega_out[t] = 1.0 + h[i] / (3.0 * rho) * drho;
        nnb_out[t] = cnt;
        divv_out[t] = -dv / rho;
        curl_out[3 * t + 0] = cx / rho;
        curl_out[3 * t + 1] = cy / rho;
        curl_out[3 * t + 2] = cz / rho;
    }
}

/* ---------------------------------------------------------------------------------------------------------
 * The fuller force view (Table 1's larger force sets: the density-loop outputs feed the force).  As or_force,
 * with the kernel family `kern`, the support kappa max(h_i, h_j), and two switchable terms:
 *   use_gradh:   P_k / rho_k^2 becomes P_k / (Omega_k rho_k^2) (the grad-h formulation, Price 2012);
 *   use_balsara: Pi_ij is multiplied by (B_i + B_j) / 2 with the Balsara (1995) switch
 *                B_k = |div v_k| / (|div v_k| + |curl v_k| + 1e-4 c_k / h_k), as in Gadget-2 (Springel 2005).
 * Also the signal velocity vsig_i = max_j (c_i + c_j - 3 min(v_ij . r_ij / r, 0)) over the same pairs (a
 * coincident pair counts c_i + c_j), 0 without neighbours.  With kern 0 and both switches off the sums are
 * or_force's (up to the rounding of the kernel's truncated-power form).
 * ------------------------------------------------------------------------------------------------------- */
void or_force_ext(int kern, int use_gradh, int use_balsara, int64_t n, const double *x, const double *v,
                  const double *m, const double *h, const double *rho, const double *P, const double *cs,
                  const double *omega, const double *divv, const double *curl, const double *box, int periodic,
                  double alpha, double beta, double eps, int64_t nt, const int64_t *targets, double *a_out,
                  double *dudt_out, double *vsig_out)
{
    double kap = or_kappa(kern);
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets[t];
        double ax = 0.0, ay = 0.0, az = 0.0, du = 0.0, vsig = 0.0;
        double Bi = 1.0;
        if (use_balsara) {
            double ci = sqrt(curl[3 * i] * curl[3 * i] + curl[3 * i + 1] * curl[3 * i + 1] +
                             curl[3 * i + 2] * curl[3 * i + 2]);
            Bi = fabs(divv[i]) / (fabs(divv[i]) + ci + 1e-4 * cs[i] / h[i]);
        }
        double Oi = use_gradh ? omega[i] : 1.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = or_min_image(x[3 * i + 0] - x[3 * j + 0], box[0], periodic);
            double dy = or_min_image(x[3 * i + 1] - x[3 * j + 1], box[1], periodic);
            double dz = or_min_image(x[3 * i + 2] - x[3 * j + 2], box[2], periodic);
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double hmax = h[i] > h[j] ? h[i] : h[j];
            if (!(r < kap * hmax)) continue;
            if (r == 0.0) {
                double vs0 = cs[i] + cs[j];
                if (vs0 > vsig) vsig = vs0;
                continue;
            }
            double gi = or_kdwdr(kern, r, h[i]) / r;
            double gj = or_kdwdr(kern, r, h[j]) / r;
            double gbar = 0.5 * (gi + gj);
            double vx = v[3 * i + 0] - v[3 * j + 0];
            double vy = v[3 * i + 1] - v[3 * j + 1];
            double vz = v[3 * i + 2] - v[3 * j + 2];
            double vdotr = vx * dx + vy * dy + vz * dz;
            double wij = vdotr / r;
            double vs = cs[i] + cs[j] - 3.0 * (wij < 0.0 ? wij : 0.0);
            if (vs > vsig) vsig = vs;
            double visc = 0.0;
            if (vdotr < 0.0) {
                double hbar = 0.5 * (h[i] + h[j]);
                double mu = hbar * vdotr / (r * r + eps * hbar * hbar);
                double cbar = 0.5 * (cs[i] + cs[j]);
                double rhobar = 0.5 * (rho[i] + rho[j]);
                visc = (-alpha * cbar * mu + beta * mu * mu) / rhobar;
                if (use_balsara) {
                    double cj = sqrt(curl[3 * j] * curl[3 * j] + curl[3 * j + 1] * curl[3 * j + 1] +
                                     curl[3 * j + 2] * curl[3 * j + 2]);
                    double Bj = fabs(divv[j]) / (fabs(divv[j]) + cj + 1e-4 * cs[j] / h[j]);
                    visc = visc * (0.5 * (Bi + Bj));
                }
            }
            double Oj = use_gradh ? omega[j] : 1.0;
            double Ai = P[i] / (Oi * rho[i] * rho[i]); /* Oi = 1: exactly P / (rho rho) */
            double Aj = P[j] / (Oj * rho[j] * rho[j]);
            double coef = m[j] * (Ai * gi + Aj * gj + visc * gbar);
            ax -= coef * dx;
            ay -= coef * dy;
            az -= coef * dz;
            du += m[j] * (Ai * gi * vdotr + 0.5 * visc * gbar * vdotr);
        }
        a_out[3 * t + 0] = ax;
        a_out[3 * t + 1] = ay;
        a_out[3 * t + 2] = az;
        dudt_out[t] = du;
        vsig_out[t] = vsig;
    }
}
