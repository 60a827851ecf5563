/*
 * Plain CPU oracle for the Radial Intersection Count Image (RICI) method.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct reference that the
 * GPU library is checked against.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load it; the product path never does.  It shares no code, header, table or
 * constant with the GPU library.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC.  Contraction must stay off so
 * every product and sum below is rounded separately, exactly as written.
 *
 * What it computes (van Blokland & Theoharis, "Radial intersection count image: a clutter
 * resistant 3D shape descriptor", 2020):
 *
 *  - oracle_rici_fp64: one N x N count image per oriented point, by brute force over every
 *    triangle of the mesh (Section 3.1: "iterate over each triangle in the scene"), in FP64:
 *      frame coefficients      Eq. rotationCoefficients (second pair read on the rotated x,
 *                              see the readings below), identity rule of Section 3.1.1
 *      projection              Eqs. relativeLocation, firstRotation, secondRotation,
 *                              calculateAlphaBeta
 *      slicing + counting      Section 3.1.2, steps 1-6 (intersection segment E0E1 of the
 *                              triangle with the plane of a circle layer; single crossings for
 *                              radii between |E0| and |E1|; double crossings between |C| and
 *                              min(|E0|,|E1|) when the closest point C lies inside the segment)
 *  - oracle_project_fp32 / oracle_rici_fp32: the same steps in single precision in one fixed
 *    operation order (see the comment above those functions), with a count of the items whose
 *    counts differ from the FP64 definition;
 *  - oracle_crss: the clutter-resistant distance of Eq. distanceFunctionExpression in int64:
 *    both images' difference images (Eq. D), then the squared differences summed where the
 *    needle's difference is non-zero.
 *  - oracle_crss_search: per needle, the distance to its true match, the rank of that match
 *    (number of haystack images strictly closer, the tie rule of Section 4.2) and the top-1
 *    haystack index (smallest index among the minimal distances).
 *  - oracle_clutter_areas: per oriented point, the surface area inside its support volume and
 *    the part of it that belongs to the object of interest (Eq. clutter), brute force over
 *    every triangle (see the comment above that function).
 *  - oracle_spin_images_fp64: spin images (Section 2.1) from m^2 point samples per triangle,
 *    FP64 positions, projection and bilinear weights summed in FP64, with a per-bin bound on
 *    the deviation of a single-precision evaluation; oracle_spin_samples /
 *    oracle_spin_images_fp32: the samples and a single-precision same-order mode with weights
 *    summed as integers in units of 2^-24 (see the comments above those functions).
 *
 * Readings where the paper is silent or garbled (each listed with its reason in the design
 * notes):
 *  (1) circle radii and layer heights sit at bin centres:
 *        alpha_c = R*(2c+1)/(2N),  beta_r = R*(2r+1-N)/(2N),  r,c in [0,N)
 *      (the support plane is R wide and R high with the spin vertex at mid-height, Sec. 2.1);
 *  (2) row r of the image is layer beta_r (ascending), column c is radius alpha_c;
 *  (3) the second normalisation acts on the rotated x component:
 *        [Nbx, Nbz] = Normalize[Nax*Snx + Nay*Sny, Snz]
 *      (Eq. secondRotation uses P''_x; the printed Normalize[Snx, Snz] only aligns the normal
 *      when Sny = 0);
 *  (4) identity rotations are (Nax,Nay) = (1,0) and (Nbx,Nbz) = (0,1);
 *  (5) a vertex is on the upper side of layer r when Tz >= beta_r; a triangle whose three
 *      vertices are on one side does not cross the layer (this also drops triangles lying
 *      inside the layer plane, the unhandled "infinite" case of Section 3.1.2);
 *  (6) intervals are half-open: single crossings for alpha^2 in (min e, max e], double
 *      crossings for alpha^2 in (|C|^2, min e], with e = |E|^2;
 *  (7) each crossed edge is evaluated from its lower-indexed vertex u to its higher-indexed
 *      vertex v (global indices), and E0 is the crossed edge with the smaller (u,v) key, so
 *      an edge shared by two triangles yields the same point in both;
 *  (8) counts saturate at 65535 (uint16 images);
 *  (9) the sums of Eq. distanceFunctionExpression run over r in [0,N) and c in [1,N).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_BAD_ARGUMENT 1
#define ORACLE_BAD_INDEX 2
#define ORACLE_NO_MEMORY 3

/* Eq. rotationCoefficients with readings (3) and (4). */
static void frame_coefficients(double nx, double ny, double nz,
                               double *Nax, double *Nay, double *Nbx, double *Nbz) {
    double h = sqrt(nx * nx + ny * ny);
    if (h == 0.0) {
        *Nax = 1.0;
        *Nay = 0.0;
    } else {
        *Nax = nx / h;
        *Nay = ny / h;
    }
    double n2x = (*Nax) * nx + (*Nay) * ny;
    double g = sqrt(n2x * n2x + nz * nz);
    if (g == 0.0) {
        *Nbx = 0.0;
        *Nbz = 1.0;
    } else {
        *Nbx = n2x / g;
        *Nbz = nz / g;
    }
}

/* Eqs. relativeLocation, firstRotation, secondRotation: T = (Tx, Ty, Tz), beta = Tz. */
static void project_point(const float *P, const double S[3], double Nax, double Nay, double Nbx,
                          double Nbz, double T[3]) {
    double px = (double)P[0] - S[0];
    double py = (double)P[1] - S[1];
    double pz = (double)P[2] - S[2];
    double qx = Nax * px + Nay * py;     /* P''_x */
    double qy = (-Nay) * px + Nax * py;  /* P''_y */
    T[0] = Nbz * qx - Nbx * pz;          /* T_x */
    T[1] = qy;                           /* T_y */
    T[2] = Nbx * qx + Nbz * pz;          /* T_z */
}

/* Section 3.1.2 step 1 for one crossed edge, evaluated from lower to higher vertex index. */
static void slice_edge(const double Tu[3], const double Tv[3], double beta, double E[2]) {
    double lambda = (beta - Tu[2]) / (Tv[2] - Tu[2]);
    E[0] = Tu[0] + lambda * (Tv[0] - Tu[0]);
    E[1] = Tu[1] + lambda * (Tv[1] - Tu[1]);
}

static int key_less(int32_t a0, int32_t a1, int32_t b0, int32_t b1) {
    return a0 < b0 || (a0 == b0 && a1 < b1);
}

/* Counts of one triangle in one layer, added to the row (steps 2-6 of Section 3.1.2). */
static void count_layer(const double T[3][3], const int32_t gid[3], double beta,
                        const double *alpha2, int32_t N, int64_t *row, int64_t *crossings,
                        int64_t *contributing) {
    int s0 = T[0][2] >= beta, s1 = T[1][2] >= beta, s2 = T[2][2] >= beta;
    if (s0 == s1 && s1 == s2) return;
    int lone = (s0 != s1 && s0 != s2) ? 0 : ((s1 != s0 && s1 != s2) ? 1 : 2);
    int oa = (lone + 1) % 3, ob = (lone + 2) % 3;
    /* the two crossed edges, each ordered by global vertex index */
    int ua = gid[lone] < gid[oa] ? lone : oa, va = gid[lone] < gid[oa] ? oa : lone;
    int ub = gid[lone] < gid[ob] ? lone : ob, vb = gid[lone] < gid[ob] ? ob : lone;
    double Ea[2], Eb[2];
    slice_edge(T[ua], T[va], beta, Ea);
    slice_edge(T[ub], T[vb], beta, Eb);
    const double *E0 = Ea, *E1 = Eb;
    if (key_less(gid[ub], gid[vb], gid[ua], gid[va])) {
        E0 = Eb;
        E1 = Ea;
    }
    (*crossings)++;
    double e0 = E0[0] * E0[0] + E0[1] * E0[1];
    double e1 = E1[0] * E1[0] + E1[1] * E1[1];
    double Dx = E1[0] - E0[0], Dy = E1[1] - E0[1];
    double d0 = E0[0] * Dx + E0[1] * Dy; /* sign: is C beyond E0 along D? */
    double d1 = E1[0] * Dx + E1[1] * Dy; /* sign: is C before E1 along D? */
    double cr = E0[0] * Dy - E0[1] * Dx; /* |C| * |D| (signed) */
    double dd = Dx * Dx + Dy * Dy;       /* |D|^2 */
    /* With both ends outside the largest circle (e >= alpha2[c] for every c) there is no
     * single crossing at any radius, and the double-crossing test alpha2[c] * dd > cr * cr can
     * only hold for some c if it holds for the largest alpha2 (rounded products are monotone):
     * such a segment, farther than alpha_{N-1} from the axis, adds nothing to the row. */
    const double amax = alpha2[N - 1];
    if (e0 >= amax && e1 >= amax && !(d0 < 0.0 && d1 > 0.0 && amax * dd > cr * cr)) return;
    (*contributing)++;
    for (int32_t c = 0; c < N; c++) {
        int in0 = e0 >= alpha2[c];
        int in1 = e1 >= alpha2[c];
        if (in0 != in1) {
            row[c] += 1;
        } else if (in0 && in1 && d0 < 0.0 && d1 > 0.0 && alpha2[c] * dd > cr * cr) {
            row[c] += 2;
        }
    }
}

int oracle_rici_fp64(const float *vertices, const float *normals, int64_t num_vertices,
                     const int32_t *triangles, int64_t num_triangles, const int32_t *origins,
                     int64_t num_origins, float support_radius, int32_t resolution,
                     uint16_t *out_images, int32_t num_threads, int64_t *counters) {
    const int32_t N = resolution;
    if (N < 1 || N > 1024 || !(support_radius > 0.0f) || num_vertices < 0 || num_triangles < 0 ||
        num_origins < 0)
        return ORACLE_BAD_ARGUMENT;
    for (int64_t t = 0; t < 3 * num_triangles; t++)
        if (triangles[t] < 0 || triangles[t] >= num_vertices) return ORACLE_BAD_INDEX;
    for (int64_t o = 0; o < num_origins; o++)
        if (origins[o] < 0 || origins[o] >= num_vertices) return ORACLE_BAD_INDEX;

    const double R = (double)support_radius;
    double *alpha2 = (double *)malloc(sizeof(double) * (size_t)N);
    double *beta = (double *)malloc(sizeof(double) * (size_t)N);
    if (!alpha2 || !beta) {
        free(alpha2);
        free(beta);
        return ORACLE_NO_MEMORY;
    }
    for (int32_t i = 0; i < N; i++) {
        double a = (R * (double)(2 * i + 1)) / (double)(2 * N);
        alpha2[i] = a * a;
        beta[i] = (R * (double)(2 * i + 1 - N)) / (double)(2 * N);
    }
    int64_t total_crossings = 0, total_pairs = 0, total_contributing = 0;
    int64_t total_contributing_pairs = 0;
    int status = ORACLE_OK;
#ifdef _OPENMP
    if (num_threads > 0) omp_set_num_threads(num_threads);
#pragma omp parallel reduction(+ : total_crossings, total_pairs, total_contributing, \
                                   total_contributing_pairs)
#endif
    {
        int64_t *img = (int64_t *)malloc(sizeof(int64_t) * (size_t)N * (size_t)N);
        /* every vertex projected once per oriented point (the same values a projection per
         * triangle corner gives) */
        double *TV = (double *)malloc(sizeof(double) * 3 * (size_t)(num_vertices > 0 ? num_vertices : 1));
        if (!img || !TV) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            status = ORACLE_NO_MEMORY;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int64_t o = 0; o < num_origins; o++) {
                memset(img, 0, sizeof(int64_t) * (size_t)N * (size_t)N);
                const int32_t sv = origins[o];
                const double S[3] = {vertices[3 * sv], vertices[3 * sv + 1], vertices[3 * sv + 2]};
                double Nax, Nay, Nbx, Nbz;
                frame_coefficients(normals[3 * sv], normals[3 * sv + 1], normals[3 * sv + 2], &Nax,
                                   &Nay, &Nbx, &Nbz);
                for (int64_t v = 0; v < num_vertices; v++)
                    project_point(vertices + 3 * v, S, Nax, Nay, Nbx, Nbz, TV + 3 * v);
                for (int64_t t = 0; t < num_triangles; t++) {
                    double T[3][3];
                    int32_t gid[3];
                    for (int k = 0; k < 3; k++) {
                        gid[k] = triangles[3 * t + k];
                        for (int d = 0; d < 3; d++) T[k][d] = TV[3 * (int64_t)gid[k] + d];
                    }
                    /* step 1's side rule for every layer at once: with all three heights
                     * below beta_0, or all at or above beta_{N-1}, no layer is crossed */
                    double zlo = T[0][2], zhi = T[0][2];
                    for (int k = 1; k < 3; k++) {
                        if (T[k][2] < zlo) zlo = T[k][2];
                        if (T[k][2] > zhi) zhi = T[k][2];
                    }
                    if (zhi < beta[0] || zlo >= beta[N - 1]) continue;
                    int64_t before = total_crossings, before_c = total_contributing;
                    /* only layers with zlo < beta_r <= zhi can be crossed; count_layer applies
                     * the side rule to each of them */
                    for (int32_t r = 0; r < N; r++) {
                        if (beta[r] <= zlo) continue;
                        if (beta[r] > zhi) break;
                        count_layer(T, gid, beta[r], alpha2, N, img + (int64_t)r * N,
                                    &total_crossings, &total_contributing);
                    }
                    if (total_crossings != before) total_pairs++;
                    if (total_contributing != before_c) total_contributing_pairs++;
                }
                uint16_t *out = out_images + o * (int64_t)N * N;
                for (int64_t b = 0; b < (int64_t)N * N; b++)
                    out[b] = (uint16_t)(img[b] > 65535 ? 65535 : img[b]);
            }
        }
        free(img);
        free(TV);
    }
    free(alpha2);
    free(beta);
    if (counters) {
        counters[0] = total_pairs;     /* (origin, triangle) pairs crossing at least one layer */
        counters[1] = total_crossings; /* (origin, triangle, layer) crossings */
        /* the same, for crossings whose segment reaches within alpha_{N-1} of the axis (the
         * ones that can add to a bin; the others are rejected by the largest circle) */
        counters[2] = total_contributing_pairs;
        counters[3] = total_contributing;
    }
    return status;
}

/* Eq. D: the horizontal difference image of one image, D(x, r, c) = x(r, c) - x(r, c-1) for
 * c in [1, N) (reading (9): the bounds of Eq. distanceFunctionExpression), stored at r*N + c;
 * entry c = 0 is left unused. */
static void difference_image(const uint16_t *x, int32_t N, int32_t *D) {
    for (int64_t p = 0; p < (int64_t)N * N; p++) {
        const int32_t c = (int32_t)(p % N);
        D[p] = c == 0 ? 0 : (int32_t)x[p] - (int32_t)x[p - 1];
    }
}

/* Eq. distanceFunctionExpression: CRD(n, h) is the sum, over the positions where the needle's
 * difference image is non-zero, of the squared difference of the two difference images
 * (positions with D(n) = 0 contribute nothing; the sum is exact in int64). */
static int64_t crd_of_differences(const int32_t *Dn, const int32_t *Dh, int32_t N) {
    int64_t total = 0;
    for (int64_t p = 0; p < (int64_t)N * N; p++) {
        if ((p % N) == 0 || Dn[p] == 0) continue;
        const int64_t e = (int64_t)Dn[p] - (int64_t)Dh[p];
        total += e * e;
    }
    return total;
}

/* Eq. distanceFunctionExpression for one pair of images. */
int64_t oracle_crss(const uint16_t *needle, const uint16_t *haystack, int32_t N) {
    int32_t *Dn = (int32_t *)malloc(sizeof(int32_t) * (size_t)N * (size_t)N);
    int32_t *Dh = (int32_t *)malloc(sizeof(int32_t) * (size_t)N * (size_t)N);
    int64_t d = -1;
    if (Dn && Dh) {
        difference_image(needle, N, Dn);
        difference_image(haystack, N, Dh);
        d = crd_of_differences(Dn, Dh, N);
    }
    free(Dn);
    free(Dh);
    return d;
}

/*
 * For every needle i: d_true[i] = CRD(needle_i, haystack[match_i]);
 * rank[i] = #{j : CRD(needle_i, haystack_j) < d_true[i]}  (Section 4.1 step 6c, ties -> best);
 * top1[i] = smallest j with the minimal distance.  distances (optional) = full Q x H matrix.
 */
int oracle_crss_search(const uint16_t *needles, int64_t num_needles, const uint16_t *haystack,
                       int64_t num_haystack, int32_t resolution, const int64_t *true_match,
                       int32_t *out_rank, int64_t *out_true_distance, int32_t *out_top1,
                       int64_t *out_distances, int32_t num_threads) {
    const int32_t N = resolution;
    if (N < 1 || num_needles < 0 || num_haystack < 0) return ORACLE_BAD_ARGUMENT;
    if (num_needles > 0 && num_haystack == 0) return ORACLE_BAD_ARGUMENT;
    for (int64_t i = 0; i < num_needles; i++) {
        int64_t m = true_match ? true_match[i] : i;
        if (m < 0 || m >= num_haystack) return ORACLE_BAD_INDEX;
    }
    const int64_t img = (int64_t)N * N;
    int status = ORACLE_OK;
#ifdef _OPENMP
    if (num_threads > 0) omp_set_num_threads(num_threads);
#pragma omp parallel
#endif
    {
        /* per thread: the needle's difference image and one haystack image's */
        int32_t *Dn = (int32_t *)malloc(sizeof(int32_t) * (size_t)img);
        int32_t *Dh = (int32_t *)malloc(sizeof(int32_t) * (size_t)img);
        if (!Dn || !Dh) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            status = ORACLE_NO_MEMORY;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int64_t i = 0; i < num_needles; i++) {
                difference_image(needles + i * img, N, Dn);
                const int64_t m = true_match ? true_match[i] : i;
                difference_image(haystack + m * img, N, Dh);
                const int64_t dt = crd_of_differences(Dn, Dh, N);
                int64_t rank = 0, best = INT64_MAX, best_j = -1;
                for (int64_t j = 0; j < num_haystack; j++) {
                    difference_image(haystack + j * img, N, Dh);
                    const int64_t d = crd_of_differences(Dn, Dh, N);
                    if (out_distances) out_distances[i * num_haystack + j] = d;
                    if (d < dt) rank++;
                    if (d < best) {
                        best = d;
                        best_j = j;
                    }
                }
                if (out_rank) out_rank[i] = (int32_t)rank;
                if (out_true_distance) out_true_distance[i] = dt;
                if (out_top1) out_top1[i] = (int32_t)best_j;
            }
        }
        free(Dn);
        free(Dh);
    }
    return status;
}

/*
 * FP32 same-operation-order mode.  The frame coefficients are the FP64 ones above, rounded to
 * float; projection, slicing and the segment quantities are evaluated in float in one fixed
 * operation order, every multiply-add written as an explicit fmaf (contraction is off, so
 * nothing else fuses):
 *   P' = P - S;  P''x = fmaf(Nay, P'y, Nax*P'x);  P''y = fmaf(Nax, P'y, -(Nay*P'x));
 *   Tx = fmaf(Nbz, P''x, -(Nbx*P'z));  Ty = P''y;  Tz = fmaf(Nbx, P''x, Nbz*P'z);
 *   a crossed edge (i, j), i < j in the triangle's own vertex order:
 *     lambda = (beta - Tz_i) * (1 / (Tz_j - Tz_i)),  E = fmaf(lambda, T_j - T_i, T_i);
 *   e = fmaf(Ex, Ex, Ey*Ey); D = E1 - E0; d0 = fmaf(E0x, Dx, E0y*Dy); d1 likewise;
 *   cr = fmaf(E0x, Dy, -(E0y*Dx)); dd = fmaf(Dx, Dx, Dy*Dy);
 * and the predicates of steps 2-6 compare them with the FP32 roundings of alpha_c^2 and beta_r.
 * E0 and E1 keep the roles of reading (7).  This is not the definition (reading (7) evaluates
 * each edge from its lower global index, in FP64); it is the arithmetic a single-precision
 * implementation of the method performs, used to measure how often single precision alone
 * would decide a count differently from the FP64 definition.
 */
static void project_point_fp32(const float *P, const float S[3], float ax, float ay, float bx,
                               float bz, float T[3]) {
    float px = P[0] - S[0], py = P[1] - S[1], pz = P[2] - S[2];
    float qx = fmaf(ay, py, ax * px);
    float qy = fmaf(ax, py, -(ay * px));
    T[0] = fmaf(bz, qx, -(bx * pz));
    T[1] = qy;
    T[2] = fmaf(bx, qx, bz * pz);
}

void oracle_project_fp32(const float *points, int64_t n, const float *spin_vertex,
                         const float *spin_normal, float *out) {
    double Nax, Nay, Nbx, Nbz;
    frame_coefficients(spin_normal[0], spin_normal[1], spin_normal[2], &Nax, &Nay, &Nbx, &Nbz);
    for (int64_t k = 0; k < n; k++)
        project_point_fp32(points + 3 * k, spin_vertex, (float)Nax, (float)Nay, (float)Nbx,
                           (float)Nbz, out + 3 * k);
}

/* Row increments of one triangle in one layer, single precision (order above). */
static int count_layer_fp32(const float T[3][3], const int32_t gid[3], float beta,
                            const float *alpha2, int32_t N, int64_t *row) {
    int s0 = T[0][2] >= beta, s1 = T[1][2] >= beta, s2 = T[2][2] >= beta;
    if (s0 == s1 && s1 == s2) return 0;
    int lone = (s0 != s1 && s0 != s2) ? 0 : ((s1 != s0 && s1 != s2) ? 1 : 2);
    int oa = lone == 0 ? 1 : 0, ob = lone == 2 ? 1 : 2;
    int ia = lone < oa ? lone : oa, ja = lone < oa ? oa : lone;
    int ib = lone < ob ? lone : ob, jb = lone < ob ? ob : lone;
    float la = (beta - T[ia][2]) * (1.0f / (T[ja][2] - T[ia][2]));
    float lb = (beta - T[ib][2]) * (1.0f / (T[jb][2] - T[ib][2]));
    float Ea[2] = {fmaf(la, T[ja][0] - T[ia][0], T[ia][0]), fmaf(la, T[ja][1] - T[ia][1], T[ia][1])};
    float Eb[2] = {fmaf(lb, T[jb][0] - T[ib][0], T[ib][0]), fmaf(lb, T[jb][1] - T[ib][1], T[ib][1])};
    int32_t ua = gid[lone] < gid[oa] ? gid[lone] : gid[oa], va = gid[lone] < gid[oa] ? gid[oa] : gid[lone];
    int32_t ub = gid[lone] < gid[ob] ? gid[lone] : gid[ob], vb = gid[lone] < gid[ob] ? gid[ob] : gid[lone];
    const float *E0 = Ea, *E1 = Eb;
    if (key_less(ub, vb, ua, va)) {
        E0 = Eb;
        E1 = Ea;
    }
    float e0 = fmaf(E0[0], E0[0], E0[1] * E0[1]);
    float e1 = fmaf(E1[0], E1[0], E1[1] * E1[1]);
    float Dx = E1[0] - E0[0], Dy = E1[1] - E0[1];
    float d0 = fmaf(E0[0], Dx, E0[1] * Dy);
    float d1 = fmaf(E1[0], Dx, E1[1] * Dy);
    float cr = fmaf(E0[0], Dy, -(E0[1] * Dx));
    float dd = fmaf(Dx, Dx, Dy * Dy);
    for (int32_t c = 0; c < N; c++) {
        int in0 = e0 >= alpha2[c], in1 = e1 >= alpha2[c];
        if (in0 != in1)
            row[c] += 1;
        else if (in0 && in1 && d0 < 0.0f && d1 > 0.0f && alpha2[c] * dd > cr * cr)
            row[c] += 2;
    }
    return 1;
}

/*
 * Images of the FP32 same-order mode, plus counters: counters[0] = (origin, triangle, layer)
 * crossings in FP32; counters[1] = items whose row increments differ between this mode and the
 * FP64 definition (the items any single-precision evaluation must send to a wider precision).
 */
int oracle_rici_fp32(const float *vertices, const float *normals, int64_t num_vertices,
                     const int32_t *triangles, int64_t num_triangles, const int32_t *origins,
                     int64_t num_origins, float support_radius, int32_t resolution,
                     uint16_t *out_images, int32_t num_threads, int64_t *counters) {
    const int32_t N = resolution;
    if (N < 1 || N > 1024 || !(support_radius > 0.0f) || num_vertices < 0 || num_triangles < 0 ||
        num_origins < 0)
        return ORACLE_BAD_ARGUMENT;
    for (int64_t t = 0; t < 3 * num_triangles; t++)
        if (triangles[t] < 0 || triangles[t] >= num_vertices) return ORACLE_BAD_INDEX;
    for (int64_t o = 0; o < num_origins; o++)
        if (origins[o] < 0 || origins[o] >= num_vertices) return ORACLE_BAD_INDEX;
    const double R = (double)support_radius;
    double *a2d = (double *)malloc(sizeof(double) * (size_t)N);
    double *bd = (double *)malloc(sizeof(double) * (size_t)N);
    float *a2f = (float *)malloc(sizeof(float) * (size_t)N);
    float *bf = (float *)malloc(sizeof(float) * (size_t)N);
    if (!a2d || !bd || !a2f || !bf) {
        free(a2d);
        free(bd);
        free(a2f);
        free(bf);
        return ORACLE_NO_MEMORY;
    }
    for (int32_t i = 0; i < N; i++) {
        double a = (R * (double)(2 * i + 1)) / (double)(2 * N);
        a2d[i] = a * a;
        bd[i] = (R * (double)(2 * i + 1 - N)) / (double)(2 * N);
        a2f[i] = (float)a2d[i];
        bf[i] = (float)bd[i];
    }
    int64_t crossings32 = 0, differing = 0;
    int status = ORACLE_OK;
#ifdef _OPENMP
    if (num_threads > 0) omp_set_num_threads(num_threads);
#pragma omp parallel reduction(+ : crossings32, differing)
#endif
    {
        int64_t *img = (int64_t *)malloc(sizeof(int64_t) * (size_t)N * (size_t)N);
        int64_t *r32 = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
        int64_t *r64 = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
        if (!img || !r32 || !r64) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            status = ORACLE_NO_MEMORY;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int64_t o = 0; o < num_origins; o++) {
                memset(img, 0, sizeof(int64_t) * (size_t)N * (size_t)N);
                const int32_t sv = origins[o];
                const float Sf[3] = {vertices[3 * sv], vertices[3 * sv + 1], vertices[3 * sv + 2]};
                const double S[3] = {Sf[0], Sf[1], Sf[2]};
                double Nax, Nay, Nbx, Nbz;
                frame_coefficients(normals[3 * sv], normals[3 * sv + 1], normals[3 * sv + 2], &Nax,
                                   &Nay, &Nbx, &Nbz);
                for (int64_t t = 0; t < num_triangles; t++) {
                    float T32[3][3];
                    double T64[3][3];
                    int32_t gid[3];
                    for (int k = 0; k < 3; k++) {
                        gid[k] = triangles[3 * t + k];
                        project_point_fp32(vertices + 3 * (int64_t)gid[k], Sf, (float)Nax,
                                           (float)Nay, (float)Nbx, (float)Nbz, T32[k]);
                        project_point(vertices + 3 * (int64_t)gid[k], S, Nax, Nay, Nbx, Nbz, T64[k]);
                    }
                    for (int32_t r = 0; r < N; r++) {
                        memset(r32, 0, sizeof(int64_t) * (size_t)N);
                        memset(r64, 0, sizeof(int64_t) * (size_t)N);
                        int64_t dummy = 0, dummy_c = 0;
                        crossings32 += count_layer_fp32(T32, gid, bf[r], a2f, N, r32);
                        count_layer(T64, gid, bd[r], a2d, N, r64, &dummy, &dummy_c);
                        if (memcmp(r32, r64, sizeof(int64_t) * (size_t)N) != 0) differing++;
                        for (int32_t c = 0; c < N; c++) img[(int64_t)r * N + c] += r32[c];
                    }
                }
                uint16_t *out = out_images + o * (int64_t)N * N;
                for (int64_t b = 0; b < (int64_t)N * N; b++)
                    out[b] = (uint16_t)(img[b] > 65535 ? 65535 : img[b]);
            }
        }
        free(img);
        free(r32);
        free(r64);
    }
    free(a2d);
    free(bd);
    free(a2f);
    free(bf);
    if (counters) {
        counters[0] = crossings32;
        counters[1] = differing;
    }
    return status;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Projection of n points into the (alpha, beta) frame of one oriented point (Section 3.1.1):
 * out[3k..3k+2] = (Tx, Ty, Tz); alpha^2 = Tx^2 + Ty^2, beta = Tz. */
void oracle_project_fp64(const float *points, int64_t n, const float *spin_vertex,
                         const float *spin_normal, double *out) {
    const double S[3] = {spin_vertex[0], spin_vertex[1], spin_vertex[2]};
    double Nax, Nay, Nbx, Nbz;
    frame_coefficients(spin_normal[0], spin_normal[1], spin_normal[2], &Nax, &Nay, &Nbx, &Nbz);
    for (int64_t k = 0; k < n; k++) project_point(points + 3 * k, S, Nax, Nay, Nbx, Nbz, out + 3 * k);
}

/* ------------------------------------------------------------------------------------------
 * Eq. clutter (Section 4.1): clutter = (A_all - A_object) / A_all, where A_all is the surface
 * area of every triangle inside the support volume of an oriented point and A_object the part
 * of it that belongs to the object of interest.
 *
 * Support volume: the cylinder swept by the image, radius R around the axis through the
 * oriented point along its normal and heights |beta| <= R/2 (readings (1) and (2) above), in
 * the frame of Eqs. relativeLocation..secondRotation: Tx^2 + Ty^2 <= R^2, |Tz| <= R/2.  The
 * projection is a rotation, so areas measured in the frame are areas in the scene.
 *
 * Per triangle: clip it to the slab |Tz| <= R/2 (a convex polygon of up to 5 vertices); the
 * part of that polygon inside the infinite cylinder is the part whose projection onto the
 * (Tx, Ty) plane lies in the disk of radius R, so its area is area(projection n disk) / |cos|,
 * with cos the z component of the triangle's unit normal.  Reading: planes with |cos| < 1e-7
 * are treated as parallel to the axis; their part inside is the polygon between the two lines
 * where the plane meets the cylinder, at the plane's mean distance from the axis.
 * A triangle belongs to the object when its first vertex index is below object_vertices (the
 * object's vertices come first).
 * ---------------------------------------------------------------------------------------- */

/* Signed area of the intersection of the triangle (0, a, b) with the disk |p| <= R: the segment
 * a-b is cut where it crosses the circle; pieces inside the disk add the triangle (0, p, q),
 * pieces outside add the circular sector between p and q. */
static double sector_piece_area(double ax, double ay, double bx, double by, double R) {
    const double dx = bx - ax, dy = by - ay;
    const double A = dx * dx + dy * dy;
    double ts[4];
    int nt = 0;
    ts[nt++] = 0.0;
    if (A > 0.0) {
        const double B = ax * dx + ay * dy;
        const double C = ax * ax + ay * ay - R * R;
        const double disc = B * B - A * C;
        if (disc > 0.0) {
            const double s = sqrt(disc);
            const double t1 = (-B - s) / A, t2 = (-B + s) / A;
            if (t1 > 0.0 && t1 < 1.0) ts[nt++] = t1;
            if (t2 > 0.0 && t2 < 1.0) ts[nt++] = t2;
        }
    }
    ts[nt++] = 1.0;
    double sum = 0.0;
    for (int i = 0; i + 1 < nt; i++) {
        const double px = ax + ts[i] * dx, py = ay + ts[i] * dy;
        const double qx = ax + ts[i + 1] * dx, qy = ay + ts[i + 1] * dy;
        const double tm = 0.5 * (ts[i] + ts[i + 1]);
        const double mx = ax + tm * dx, my = ay + tm * dy;
        const double cross = px * qy - py * qx;
        if (mx * mx + my * my <= R * R)
            sum += 0.5 * cross;
        else
            sum += 0.5 * R * R * atan2(cross, px * qx + py * qy);
    }
    return sum;
}

/* Sutherland-Hodgman step: keep the part of the polygon where sign * z <= lim. */
static int clip_height(const double (*in)[3], int n, double (*out)[3], double sign, double lim) {
    int m = 0;
    for (int i = 0; i < n; i++) {
        const double *P = in[i], *Q = in[(i + 1) % n];
        const double dp = lim - sign * P[2], dq = lim - sign * Q[2];
        if (dp >= 0.0) {
            out[m][0] = P[0];
            out[m][1] = P[1];
            out[m][2] = P[2];
            m++;
        }
        if ((dp >= 0.0) != (dq >= 0.0)) {
            const double t = dp / (dp - dq);
            for (int k = 0; k < 3; k++) out[m][k] = P[k] + t * (Q[k] - P[k]);
            m++;
        }
    }
    return m;
}

/* Keep the part of a 2D polygon where sign * h <= lim. */
static int clip_line(const double (*in)[2], int n, double (*out)[2], double sign, double lim) {
    int m = 0;
    for (int i = 0; i < n; i++) {
        const double *P = in[i], *Q = in[(i + 1) % n];
        const double dp = lim - sign * P[0], dq = lim - sign * Q[0];
        if (dp >= 0.0) {
            out[m][0] = P[0];
            out[m][1] = P[1];
            m++;
        }
        if ((dp >= 0.0) != (dq >= 0.0)) {
            const double t = dp / (dp - dq);
            out[m][0] = P[0] + t * (Q[0] - P[0]);
            out[m][1] = P[1] + t * (Q[1] - P[1]);
            m++;
        }
    }
    return m;
}

/* Area of the part of one projected triangle inside the support volume. */
static double support_area(const double T[3][3], double R) {
    const double ux = T[1][0] - T[0][0], uy = T[1][1] - T[0][1], uz = T[1][2] - T[0][2];
    const double vx = T[2][0] - T[0][0], vy = T[2][1] - T[0][1], vz = T[2][2] - T[0][2];
    const double nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
    const double nn = sqrt(nx * nx + ny * ny + nz * nz);
    if (nn == 0.0) return 0.0;
    double a[6][3], b[6][3];
    for (int k = 0; k < 3; k++)
        for (int j = 0; j < 3; j++) a[k][j] = T[k][j];
    int m = clip_height((const double(*)[3])a, 3, b, 1.0, 0.5 * R);
    if (m < 3) return 0.0;
    m = clip_height((const double(*)[3])b, m, a, -1.0, 0.5 * R);
    if (m < 3) return 0.0;
    const double cz = fabs(nz) / nn;
    if (cz >= 1e-7) {
        double s = 0.0;
        for (int i = 0; i < m; i++)
            s += sector_piece_area(a[i][0], a[i][1], a[(i + 1) % m][0], a[(i + 1) % m][1], R);
        return fabs(s) / cz;
    }
    /* plane parallel to the axis: in-plane coordinates (h along the horizontal direction of
     * the plane, z), inside where |h| <= sqrt(R^2 - p^2), p = distance of the plane from the
     * axis */
    const double hxy = sqrt(nx * nx + ny * ny);
    const double ex = -ny / hxy, ey = nx / hxy, wx = nx / hxy, wy = ny / hxy;
    double p = 0.0;
    for (int i = 0; i < m; i++) p += a[i][0] * wx + a[i][1] * wy;
    p /= (double)m;
    if (fabs(p) >= R) return 0.0;
    const double c = sqrt(R * R - p * p);
    double h[7][2], g[7][2];
    for (int i = 0; i < m; i++) {
        h[i][0] = a[i][0] * ex + a[i][1] * ey;
        h[i][1] = a[i][2];
    }
    int k = clip_line((const double(*)[2])h, m, g, 1.0, c);
    if (k < 3) return 0.0;
    k = clip_line((const double(*)[2])g, k, h, -1.0, c);
    if (k < 3) return 0.0;
    double s = 0.0;
    for (int i = 0; i < k; i++) s += h[i][0] * h[(i + 1) % k][1] - h[(i + 1) % k][0] * h[i][1];
    return 0.5 * fabs(s);
}

/* Per origin: area_all[o] = A_all, area_object[o] = A_object (brute force over all triangles). */
int oracle_clutter_areas(const float *vertices, const float *normals, int64_t num_vertices,
                         const int32_t *triangles, int64_t num_triangles, const int32_t *origins,
                         int64_t num_origins, float support_radius, int64_t object_vertices,
                         double *area_all, double *area_object, int32_t num_threads) {
    if (!(support_radius > 0.0f) || num_vertices < 0 || num_triangles < 0 || num_origins < 0)
        return ORACLE_BAD_ARGUMENT;
    for (int64_t t = 0; t < 3 * num_triangles; t++)
        if (triangles[t] < 0 || triangles[t] >= num_vertices) return ORACLE_BAD_INDEX;
    for (int64_t o = 0; o < num_origins; o++)
        if (origins[o] < 0 || origins[o] >= num_vertices) return ORACLE_BAD_INDEX;
    const double R = (double)support_radius;
#ifdef _OPENMP
    if (num_threads > 0) omp_set_num_threads(num_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t o = 0; o < num_origins; o++) {
        const int32_t sv = origins[o];
        const double S[3] = {vertices[3 * sv], vertices[3 * sv + 1], vertices[3 * sv + 2]};
        double Nax, Nay, Nbx, Nbz;
        frame_coefficients(normals[3 * sv], normals[3 * sv + 1], normals[3 * sv + 2], &Nax, &Nay,
                           &Nbx, &Nbz);
        double all = 0.0, obj = 0.0;
        for (int64_t t = 0; t < num_triangles; t++) {
            double T[3][3];
            for (int k = 0; k < 3; k++)
                project_point(vertices + 3 * (int64_t)triangles[3 * t + k], S, Nax, Nay, Nbx, Nbz,
                              T[k]);
            const double a = support_area((const double(*)[3])T, R);
            all += a;
            if (triangles[3 * t] < object_vertices) obj += a;
        }
        area_all[o] = all;
        area_object[o] = obj;
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------------------------
 * Spin images (Section 2.1: the descriptor the RICI is compared with), generated from point
 * samples of the mesh with the projection of Section 3.1.1.  oracle_spin_images_fp64 (further
 * below) is the definition; oracle_spin_images_fp32 is a single-precision same-operation-order
 * mode, a second check of a GPU evaluation's arithmetic, itself pinned to the FP64 definition.
 *
 * Samples: m^2 points per triangle (A, B, C in its own vertex order), the centroids of the m^2
 * congruent triangles obtained by dividing every side into m parts, so the samples are spread
 * uniformly over the triangle's area.  With barycentric weights (a, b) for B and C:
 *   upward sub-triangles   i + j <= m - 1:  a = (3i + 1) / (3m),  b = (3j + 1) / (3m)
 *   downward sub-triangles i + j <= m - 2:  a = (3i + 2) / (3m),  b = (3j + 2) / (3m)
 *   P = fmaf(b, C - A, fmaf(a, B - A, A)) per coordinate (float).
 * Readings: the square plane is R wide and R high with its left side on the central axis and
 * the spin vertex at half height (Section 2.1), divided into N x N bins centred at
 * (alpha_c, beta_r) of readings (1)-(2); a sample with alpha^2 < R^2 and -R/2 <= beta < R/2 is
 * in the support volume and adds bilinear weights (Section 2.1) to the four bins around it:
 *   u = alpha N/R - 1/2, v = (beta + R/2) N/R - 1/2, c = floor(u), r = floor(v),
 *   fu = u - c, fv = v - r: (1-fu)(1-fv) to (r, c), fu (1-fv) to (r, c+1), (1-fu) fv to
 *   (r+1, c), fu fv to (r+1, c+1); weight that falls on a bin outside [0, N) is dropped.
 * The support-angle filter is not applied (Section 4.2 found it does not help).
 * FP32 mode: every float operation is written out in one fixed order (projection as
 * oracle_project_fp32), and each weight is accumulated as an integer number of units of 2^-24
 * (w * 2^24 rounded to the nearest integer), so a bin's sum is exact and does not depend on the
 * order of the samples; the image stores float32(sum * 2^-24).  This quantisation belongs to
 * the single-precision mode only, not to the definition.
 * ---------------------------------------------------------------------------------------- */

/* Barycentric weights (a, b) of sample k of m^2 (upward sub-triangles first). */
static void spin_sample_weights(int m, int k, float *a, float *b) {
    const int up = m * (m + 1) / 2;
    const float den = (float)(3 * m);
    int idx = k < up ? k : k - up;
    const int off = k < up ? 1 : 2;
    const int rows = k < up ? m : m - 1;
    int i = 0;
    while (idx >= rows - i) {
        idx -= rows - i;
        i++;
    }
    const int j = idx;
    *a = (float)(3 * i + off) / den;
    *b = (float)(3 * j + off) / den;
}

/* Sample positions of every triangle: out[t][k][3], m^2 samples per triangle. */
int oracle_spin_samples(const float *vertices, int64_t num_vertices, const int32_t *triangles,
                        int64_t num_triangles, int32_t m, float *out) {
    if (m < 1 || m > 16 || num_triangles < 0) return ORACLE_BAD_ARGUMENT;
    for (int64_t t = 0; t < 3 * num_triangles; t++)
        if (triangles[t] < 0 || triangles[t] >= num_vertices) return ORACLE_BAD_INDEX;
    for (int64_t t = 0; t < num_triangles; t++) {
        const float *A = vertices + 3 * (int64_t)triangles[3 * t];
        const float *B = vertices + 3 * (int64_t)triangles[3 * t + 1];
        const float *C = vertices + 3 * (int64_t)triangles[3 * t + 2];
        for (int k = 0; k < m * m; k++) {
            float a, b;
            spin_sample_weights(m, k, &a, &b);
            float *P = out + (t * (int64_t)m * m + k) * 3;
            for (int d = 0; d < 3; d++) P[d] = fmaf(b, C[d] - A[d], fmaf(a, B[d] - A[d], A[d]));
        }
    }
    return ORACLE_OK;
}

int oracle_spin_images_fp32(const float *vertices, const float *normals, int64_t num_vertices,
                            const int32_t *triangles, int64_t num_triangles,
                            const int32_t *origins, int64_t num_origins, float support_radius,
                            int32_t resolution, int32_t m, float *out_images,
                            int32_t num_threads) {
    const int32_t N = resolution;
    if (N < 1 || N > 1024 || m < 1 || m > 16 || !(support_radius > 0.0f) || num_vertices < 0 ||
        num_triangles < 0 || num_origins < 0)
        return ORACLE_BAD_ARGUMENT;
    for (int64_t t = 0; t < 3 * num_triangles; t++)
        if (triangles[t] < 0 || triangles[t] >= num_vertices) return ORACLE_BAD_INDEX;
    for (int64_t o = 0; o < num_origins; o++)
        if (origins[o] < 0 || origins[o] >= num_vertices) return ORACLE_BAD_INDEX;
    const float R = support_radius;
    const float R2 = R * R, H = 0.5f * R, s = (float)N / R;
    int status = ORACLE_OK;
#ifdef _OPENMP
    if (num_threads > 0) omp_set_num_threads(num_threads);
#pragma omp parallel
#endif
    {
        uint64_t *img = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N * (size_t)N);
        if (!img) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            status = ORACLE_NO_MEMORY;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int64_t o = 0; o < num_origins; o++) {
                memset(img, 0, sizeof(uint64_t) * (size_t)N * (size_t)N);
                const int32_t sv = origins[o];
                const float S[3] = {vertices[3 * sv], vertices[3 * sv + 1], vertices[3 * sv + 2]};
                double Nax, Nay, Nbx, Nbz;
                frame_coefficients(normals[3 * sv], normals[3 * sv + 1], normals[3 * sv + 2],
                                   &Nax, &Nay, &Nbx, &Nbz);
                const float ax = (float)Nax, ay = (float)Nay, bx = (float)Nbx, bz = (float)Nbz;
                for (int64_t t = 0; t < num_triangles; t++) {
                    const float *A = vertices + 3 * (int64_t)triangles[3 * t];
                    const float *B = vertices + 3 * (int64_t)triangles[3 * t + 1];
                    const float *C = vertices + 3 * (int64_t)triangles[3 * t + 2];
                    for (int k = 0; k < m * m; k++) {
                        float a, b, P[3], T[3];
                        spin_sample_weights(m, k, &a, &b);
                        for (int d = 0; d < 3; d++)
                            P[d] = fmaf(b, C[d] - A[d], fmaf(a, B[d] - A[d], A[d]));
                        project_point_fp32(P, S, ax, ay, bx, bz, T);
                        const float a2 = fmaf(T[0], T[0], T[1] * T[1]);
                        if (!(a2 < R2) || !(T[2] >= -H) || !(T[2] < H)) continue;
                        const float u = fmaf(sqrtf(a2), s, -0.5f);
                        const float v = fmaf(T[2] + H, s, -0.5f);
                        const float cu = floorf(u), rv = floorf(v);
                        const float fu = u - cu, fv = v - rv;
                        const int c = (int)cu, r = (int)rv;
                        const float w[4] = {(1.0f - fu) * (1.0f - fv), fu * (1.0f - fv),
                                            (1.0f - fu) * fv, fu * fv};
                        for (int q = 0; q < 4; q++) {
                            const int rr = r + (q >> 1), cc = c + (q & 1);
                            if (rr >= 0 && rr < N && cc >= 0 && cc < N)
                                img[(int64_t)rr * N + cc] += (uint64_t)rintf(w[q] * 16777216.0f);
                        }
                    }
                }
                float *dst = out_images + o * (int64_t)N * N;
                for (int64_t k = 0; k < (int64_t)N * N; k++)
                    dst[k] = (float)((double)img[k] * (1.0 / 16777216.0));
            }
            free(img);
        }
    }
    return status;
}

/* ------------------------------------------------------------------------------------------
 * Spin images in FP64: the definition of Section 2.1 with the sample pattern above, evaluated
 * in double precision throughout and summed as real numbers.
 *
 *   samples   P = A + a (B - A) + b (C - A) with the barycentric weights a = (3i + off)/(3m),
 *             b = (3j + off)/(3m) of oracle_spin_samples, in double;
 *   frame     Eq. rotationCoefficients in double (frame_coefficients);
 *   projection Eqs. relativeLocation, firstRotation, secondRotation in double (project_point's
 *             arithmetic on the double sample);
 *   volume    alpha^2 < R^2 and -R/2 <= beta < R/2;
 *   weights   bilinear around the bin centres (readings (1)-(2)): u = alpha N/R - 1/2,
 *             v = (beta + R/2) N/R - 1/2, (1-fu)(1-fv), fu(1-fv), (1-fu)fv, fu fv on the bins
 *             (r, c), (r, c+1), (r+1, c), (r+1, c+1), c = floor(u), r = floor(v); weight on a bin
 *             outside the image is dropped;
 *   image     the double sum of the weights, rounded once to float.
 *
 * out_bound (optional, [O][N][N] double) receives, per bin, a bound on how far an evaluation of
 * the same definition in single precision may lie from this image: each sample position, the
 * projection, alpha = sqrt(Tx^2 + Ty^2), u and v formed in FP32 (one rounding per operation,
 * fused multiply-adds where the single-precision form uses them, the frame coefficients rounded
 * from FP64 to FP32), each weight rounded to a multiple of 2^-24, and the bin sums rounded to
 * float.  For one sample, with unit roundoff u32 = 2^-24:
 *   dP_d  <= u32 (|P_d| + |A_d + a (B_d - A_d)| + 2 a |B_d - A_d| + 2 b |C_d - A_d|)
 *            (a and b rounded, B - A and C - A rounded, two fused multiply-adds);
 *   dT    <= 10 u32 (|d_x| + |d_y| + |d_z|) + sum_d dP_d with d = P - S (the projection bound of
 *            the FP32 mode, pinned by the tests, plus the position error carried through the
 *            rotation, whose rows have unit length);
 *   dA2   <= 2 (|Tx| + |Ty|) dT + 2 dT^2 + 2 u32 alpha^2  (alpha^2 = Tx^2 + Ty^2);
 *   dAl   <= min(sqrt(dA2), dA2 / alpha) + u32 alpha;
 *   du    <= s dAl + 2 u32 s alpha + u32 |u|,  s = N/R;
 *   dv    <= s (dT + u32 |beta + R/2|) + u32 s |beta + R/2| + u32 |v|;
 *   dw    <= du + dv + du dv + 3 u32 + 2^-25  (|d w / d fu| <= 1 and |d w / d fv| <= 1; two
 *            roundings in 1 - f and one in the product; the 2^-24 quantisation).
 * Twice dw is added to every bin the sample can reach in either evaluation (floor(u - du) ..
 * floor(u + du) + 1, and the same for v).  A sample that may fall on the other side of the
 * volume boundary in single precision (|alpha^2 - R^2| <= 2 (dA2 + u32 R^2), or beta within
 * 2 dT of -R/2 or R/2) adds 1 (the largest weight) to each bin it can reach instead.  Finally
 * 2^-23 |image| covers the two roundings of a bin sum to float.
 * ---------------------------------------------------------------------------------------- */
static void spin_sample_index(int m, int k, int *i_out, int *j_out, int *off_out) {
    const int up = m * (m + 1) / 2;
    int idx = k < up ? k : k - up;
    const int rows = k < up ? m : m - 1;
    int i = 0;
    while (idx >= rows - i) {
        idx -= rows - i;
        i++;
    }
    *i_out = i;
    *j_out = idx;
    *off_out = k < up ? 1 : 2;
}

int oracle_spin_images_fp64(const float *vertices, const float *normals, int64_t num_vertices,
                            const int32_t *triangles, int64_t num_triangles,
                            const int32_t *origins, int64_t num_origins, float support_radius,
                            int32_t resolution, int32_t m, float *out_images, double *out_bound,
                            int32_t num_threads) {
    const int32_t N = resolution;
    if (N < 1 || N > 1024 || m < 1 || m > 16 || !(support_radius > 0.0f) || num_vertices < 0 ||
        num_triangles < 0 || num_origins < 0)
        return ORACLE_BAD_ARGUMENT;
    for (int64_t t = 0; t < 3 * num_triangles; t++)
        if (triangles[t] < 0 || triangles[t] >= num_vertices) return ORACLE_BAD_INDEX;
    for (int64_t o = 0; o < num_origins; o++)
        if (origins[o] < 0 || origins[o] >= num_vertices) return ORACLE_BAD_INDEX;
    const double R = (double)support_radius;
    const double R2 = R * R, H = 0.5 * R, s = (double)N / R;
    const double u32 = 1.0 / 16777216.0;
    const int64_t NN = (int64_t)N * N;
    int status = ORACLE_OK;
#ifdef _OPENMP
    if (num_threads > 0) omp_set_num_threads(num_threads);
#pragma omp parallel
#endif
    {
        double *img = (double *)malloc(sizeof(double) * (size_t)NN);
        double *bnd = (double *)malloc(sizeof(double) * (size_t)NN);
        if (!img || !bnd) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            status = ORACLE_NO_MEMORY;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int64_t o = 0; o < num_origins; o++) {
                memset(img, 0, sizeof(double) * (size_t)NN);
                memset(bnd, 0, sizeof(double) * (size_t)NN);
                const int32_t sv = origins[o];
                const double S[3] = {vertices[3 * sv], vertices[3 * sv + 1], vertices[3 * sv + 2]};
                double Nax, Nay, Nbx, Nbz;
                frame_coefficients(normals[3 * sv], normals[3 * sv + 1], normals[3 * sv + 2],
                                   &Nax, &Nay, &Nbx, &Nbz);
                for (int64_t t = 0; t < num_triangles; t++) {
                    const float *A = vertices + 3 * (int64_t)triangles[3 * t];
                    const float *B = vertices + 3 * (int64_t)triangles[3 * t + 1];
                    const float *C = vertices + 3 * (int64_t)triangles[3 * t + 2];
                    for (int k = 0; k < m * m; k++) {
                        int si, sj, off;
                        spin_sample_index(m, k, &si, &sj, &off);
                        const double a = (double)(3 * si + off) / (double)(3 * m);
                        const double b = (double)(3 * sj + off) / (double)(3 * m);
                        double P[3], dP = 0.0, dsum = 0.0;
                        for (int d = 0; d < 3; d++) {
                            const double ba = (double)B[d] - (double)A[d];
                            const double ca = (double)C[d] - (double)A[d];
                            const double inner = (double)A[d] + a * ba;
                            P[d] = inner + b * ca;
                            dP += u32 * (fabs(P[d]) + fabs(inner) + 2.0 * a * fabs(ba) +
                                         2.0 * b * fabs(ca));
                            dsum += fabs(P[d] - S[d]);
                        }
                        /* Eqs. relativeLocation, firstRotation, secondRotation */
                        const double px = P[0] - S[0], py = P[1] - S[1], pz = P[2] - S[2];
                        const double qx = Nax * px + Nay * py;
                        const double qy = (-Nay) * px + Nax * py;
                        const double Tx = Nbz * qx - Nbx * pz;
                        const double Ty = qy;
                        const double Tz = Nbx * qx + Nbz * pz;
                        const double alpha2 = Tx * Tx + Ty * Ty;
                        const int inside = alpha2 < R2 && Tz >= -H && Tz < H;
                        /* single-precision deviation of this sample (comment above) */
                        const double dT = 10.0 * u32 * dsum + dP;
                        const double dA2 = 2.0 * (fabs(Tx) + fabs(Ty)) * dT + 2.0 * dT * dT +
                                           2.0 * u32 * alpha2;
                        const double alpha = sqrt(alpha2);
                        double dAl = sqrt(dA2);
                        if (alpha > 0.0 && dA2 / alpha < dAl) dAl = dA2 / alpha;
                        dAl += u32 * alpha;
                        const double u = alpha * s - 0.5;
                        const double v = (Tz + H) * s - 0.5;
                        const double du = s * dAl + 2.0 * u32 * s * alpha + u32 * fabs(u);
                        const double dv = s * (dT + u32 * fabs(Tz + H)) +
                                          u32 * s * fabs(Tz + H) + u32 * fabs(v);
                        const double dw = du + dv + du * dv + 3.0 * u32 + 0.5 * u32;
                        const int flip = fabs(alpha2 - R2) <= 2.0 * (dA2 + u32 * R2) ||
                                         fabs(Tz + H) <= 2.0 * dT || fabs(Tz - H) <= 2.0 * dT;
                        if (inside) {
                            const double cu = floor(u), rv = floor(v);
                            const double fu = u - cu, fv = v - rv;
                            const int c = (int)cu, r = (int)rv;
                            const double w[4] = {(1.0 - fu) * (1.0 - fv), fu * (1.0 - fv),
                                                 (1.0 - fu) * fv, fu * fv};
                            for (int q = 0; q < 4; q++) {
                                const int rr = r + (q >> 1), cc = c + (q & 1);
                                if (rr >= 0 && rr < N && cc >= 0 && cc < N)
                                    img[(int64_t)rr * N + cc] += w[q];
                            }
                        }
                        if (out_bound && (inside || flip)) {
                            /* bins the sample can reach in either evaluation */
                            const double add = flip ? 1.0 : 2.0 * dw;
                            int c_lo = (int)floor(u - du), c_hi = (int)floor(u + du) + 1;
                            int r_lo = (int)floor(v - dv), r_hi = (int)floor(v + dv) + 1;
                            if (c_lo < 0) c_lo = 0;
                            if (r_lo < 0) r_lo = 0;
                            if (c_hi > N - 1) c_hi = N - 1;
                            if (r_hi > N - 1) r_hi = N - 1;
                            for (int rr = r_lo; rr <= r_hi; rr++)
                                for (int cc = c_lo; cc <= c_hi; cc++)
                                    bnd[(int64_t)rr * N + cc] += add;
                        }
                    }
                }
                float *dst = out_images + o * NN;
                for (int64_t q = 0; q < NN; q++) dst[q] = (float)img[q];
                if (out_bound) {
                    double *db = out_bound + o * NN;
                    for (int64_t q = 0; q < NN; q++)
                        db[q] = bnd[q] + fabs(img[q]) * (2.0 * u32) + 1e-30;
                }
            }
        }
        free(img);
        free(bnd);
    }
    return status;
}
