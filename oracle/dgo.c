/*
 * dgo.c -- plain, slow, FP64 CPU oracle of the differentiable tile rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library in paper_2503_18402_gb300/) never calls it, shares no
 * code, header, table or constant generator with it, and fails loudly when
 * its own CUDA extension is missing.
 *
 * What it computes (DashGaussian, Sec. 3 "Preliminary", Eq. 1, with the 3DGS
 * backbone rasterizer the paper keeps unchanged, Sec. 5 "Implementation
 * Details"):
 *   - projection of each 3D Gaussian (centre p, covariance from scale and
 *     rotation, opacity o, colour coefficients c) to a 2D Gaussian on the
 *     image plane (local affine / EWA approximation of the perspective map);
 *   - real spherical-harmonic colour up to degree 3;
 *   - tile binning and the (tile, depth, index) order of each tile's list;
 *   - front-to-back alpha compositing, Eq. 1: C(u) = sum_i T_i w_i c_i,
 *     T_i = prod_{j<i} (1 - w_j), w_i = o_i G2D_i(u), plus background T_N bg;
 *   - the exact adjoint of all of the above ("fully differentiable", Sec. 3);
 *   - the L1 loss and the Adam update (Kingma & Ba) of the 3DGS backbone.
 *
 * Readings where the paper is silent (the same readings bind the CUDA path):
 *   near plane 0.2; 2D dilation eps = 0.3 px^2; frustum guard 1.3 x half-FOV
 *   tangent on the Jacobian only (exact derivative of the clamped map);
 *   radius = ceil(3 sqrt(lambda_max)); pixel (x, y) sampled at (x+.5, y+.5);
 *   tile rect [floor((u-r)/B), floor((u+r)/B)+1) clipped to the grid;
 *   alpha = min(0.99, o exp(power)), skip power > 0 and alpha < 1/255,
 *   stop before blending when T (1 - alpha) < 1e-4; colour = SH + 0.5 clamped
 *   at 0.  Per-Gaussian parameter rows (59 values): mean[3], log_scale[3],
 *   quaternion (w,x,y,z)[4], opacity logit[1], SH[16][3] (coefficient-major).
 *
 * Plain code on purpose: no blocking, no fusion, no reordering.  The
 * backward pass stores every blended (pixel, Gaussian) pair instead of
 * recomputing transmittance by division.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { NP = 59, O_MEAN = 0, O_LSCALE = 3, O_QUAT = 6, O_OPAC = 10, O_SH = 11 };
enum { NF = 9 }; /* feature record: u v A B C o r g b */

typedef struct dgo_consts {
    double near_plane;    /* cull when camera-space z <= near_plane */
    double eps2d;         /* low-pass dilation added to the 2D covariance */
    double alpha_max;     /* alpha clamp */
    double alpha_min;     /* skip a Gaussian whose alpha is below this */
    double t_min;         /* stop before blending when T would fall below */
    double frustum_guard; /* clamp of t_x/t_z in the Jacobian, x half-FOV tan */
    int32_t tile;         /* tile edge B in pixels */
    int32_t sh_degree;    /* 0..3 */
    double mip2d;         /* > 0: Mip-Splatting 2D filter of this variance in place of the
                             dilation, opacity scaled by sqrt(det(S2) / det(S2 + mip2d I)) */
} dgo_consts;

typedef struct dgo_camera {
    double R[9];  /* world-to-camera rotation, row-major */
    double t[3];  /* world-to-camera translation: x_cam = R x + t */
    double fx, fy, cx, cy;
    int32_t width, height;
} dgo_camera;

/* ------------------------------------------------------------------ */
/* Real spherical harmonics, orthonormal on the unit sphere, degree <= 3,
 * index k = l*l + l + m.  Written from the Cartesian polynomial forms of
 * the real SH (no Condon-Shortley phase).  grad[k][3] is the gradient of
 * the polynomial in (x, y, z); only its tangential part matters because
 * the direction is normalised. */
static void sh_basis(const double d[3], double Y[16], double G[16][3])
{
    const double x = d[0], y = d[1], z = d[2];
    const double pi = 3.14159265358979323846;
    const double c0 = 0.5 * sqrt(1.0 / pi);
    const double c1 = sqrt(3.0 / (4.0 * pi));
    const double c2a = 0.5 * sqrt(15.0 / pi);      /* xy, yz, xz */
    const double c20 = 0.25 * sqrt(5.0 / pi);      /* 3z^2 - 1 */
    const double c22 = 0.25 * sqrt(15.0 / pi);     /* x^2 - y^2 */
    const double c33 = 0.25 * sqrt(35.0 / (2.0 * pi));
    const double c32a = 0.5 * sqrt(105.0 / pi);    /* xyz */
    const double c31 = 0.25 * sqrt(21.0 / (2.0 * pi));
    const double c30 = 0.25 * sqrt(7.0 / pi);
    const double c32b = 0.25 * sqrt(105.0 / pi);   /* z (x^2 - y^2) */
    memset(G, 0, sizeof(double) * 48);
    Y[0] = c0;
    Y[1] = c1 * y;  G[1][1] = c1;
    Y[2] = c1 * z;  G[2][2] = c1;
    Y[3] = c1 * x;  G[3][0] = c1;
    Y[4] = c2a * x * y;  G[4][0] = c2a * y;  G[4][1] = c2a * x;
    Y[5] = c2a * y * z;  G[5][1] = c2a * z;  G[5][2] = c2a * y;
    Y[6] = c20 * (3.0 * z * z - 1.0);  G[6][2] = c20 * 6.0 * z;
    Y[7] = c2a * x * z;  G[7][0] = c2a * z;  G[7][2] = c2a * x;
    Y[8] = c22 * (x * x - y * y);  G[8][0] = c22 * 2.0 * x;  G[8][1] = -c22 * 2.0 * y;
    Y[9] = c33 * y * (3.0 * x * x - y * y);
    G[9][0] = c33 * 6.0 * x * y;  G[9][1] = c33 * (3.0 * x * x - 3.0 * y * y);
    Y[10] = c32a * x * y * z;
    G[10][0] = c32a * y * z;  G[10][1] = c32a * x * z;  G[10][2] = c32a * x * y;
    Y[11] = c31 * y * (5.0 * z * z - 1.0);
    G[11][1] = c31 * (5.0 * z * z - 1.0);  G[11][2] = c31 * 10.0 * y * z;
    Y[12] = c30 * z * (5.0 * z * z - 3.0);  G[12][2] = c30 * (15.0 * z * z - 3.0);
    Y[13] = c31 * x * (5.0 * z * z - 1.0);
    G[13][0] = c31 * (5.0 * z * z - 1.0);  G[13][2] = c31 * 10.0 * x * z;
    Y[14] = c32b * z * (x * x - y * y);
    G[14][0] = c32b * 2.0 * x * z;  G[14][1] = -c32b * 2.0 * y * z;  G[14][2] = c32b * (x * x - y * y);
    Y[15] = c33 * x * (x * x - 3.0 * y * y);
    G[15][0] = c33 * (3.0 * x * x - 3.0 * y * y);  G[15][1] = -c33 * 6.0 * x * y;
}

void dgo_sh_basis(const double* dirs, int64_t n, double* out16)
{
    double G[16][3];
    for (int64_t i = 0; i < n; ++i) sh_basis(dirs + 3 * i, out16 + 16 * i, G);
}

/* ------------------------------------------------------------------ */
/* Per-Gaussian projection with every intermediate kept for the adjoint. */
typedef struct gproj {
    int visible;
    double p[3], t[3];
    double q[4], qlen, qn[4];
    double Rq[9], s[3], M[9], Sig[9];
    int clampx, clampy;
    double limx, limy;   /* signed clamp value of t_x/t_z, t_y/t_z when active */
    double J[6], T2[6];
    double a, b, c, det, conic[3];
    double u, v;
    int64_t radius;
    int64_t rect[4];
    double campos[3], draw[3], dlen, dir[3];
    double rgb[3];
    int clamp[3];
    double osig;          /* sigmoid of the opacity logit */
    double det0, comp;    /* 2D-filter opacity compensation sqrt(det0 / det) (1 without it) */
    double o;             /* opacity of the record: osig * comp */
} gproj;

static int64_t floordiv(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) --q;
    return q;
}

static void project_one(const double* g, const dgo_camera* cam, const dgo_consts* k, gproj* P)
{
    memset(P, 0, sizeof *P);
    const double* R = cam->R;
    for (int i = 0; i < 3; ++i) P->p[i] = g[O_MEAN + i];
    for (int i = 0; i < 3; ++i)
        P->t[i] = R[3 * i] * P->p[0] + R[3 * i + 1] * P->p[1] + R[3 * i + 2] * P->p[2] + cam->t[i];
    const double tx = P->t[0], ty = P->t[1], tz = P->t[2];
    if (!(tz > k->near_plane)) return;

    /* rotation from the normalised quaternion (w, x, y, z) */
    for (int i = 0; i < 4; ++i) P->q[i] = g[O_QUAT + i];
    P->qlen = sqrt(P->q[0] * P->q[0] + P->q[1] * P->q[1] + P->q[2] * P->q[2] + P->q[3] * P->q[3]);
    for (int i = 0; i < 4; ++i) P->qn[i] = P->q[i] / P->qlen;
    const double w = P->qn[0], x = P->qn[1], y = P->qn[2], z = P->qn[3];
    double* Rq = P->Rq;
    Rq[0] = 1.0 - 2.0 * (y * y + z * z); Rq[1] = 2.0 * (x * y - w * z);       Rq[2] = 2.0 * (x * z + w * y);
    Rq[3] = 2.0 * (x * y + w * z);       Rq[4] = 1.0 - 2.0 * (x * x + z * z); Rq[5] = 2.0 * (y * z - w * x);
    Rq[6] = 2.0 * (x * z - w * y);       Rq[7] = 2.0 * (y * z + w * x);       Rq[8] = 1.0 - 2.0 * (x * x + y * y);
    for (int i = 0; i < 3; ++i) P->s[i] = exp(g[O_LSCALE + i]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P->M[3 * i + j] = Rq[3 * i + j] * P->s[j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int l = 0; l < 3; ++l) acc += P->M[3 * i + l] * P->M[3 * j + l];
            P->Sig[3 * i + j] = acc;
        }

    /* Jacobian of the perspective map at the (guarded) mean */
    const double lx = k->frustum_guard * 0.5 * cam->width / cam->fx;
    const double ly = k->frustum_guard * 0.5 * cam->height / cam->fy;
    double txtz = tx / tz, tytz = ty / tz;
    double txc = tx, tyc = ty;
    if (txtz < -lx || txtz > lx) { P->clampx = 1; P->limx = txtz < 0 ? -lx : lx; txc = P->limx * tz; }
    if (tytz < -ly || tytz > ly) { P->clampy = 1; P->limy = tytz < 0 ? -ly : ly; tyc = P->limy * tz; }
    double* J = P->J;
    J[0] = cam->fx / tz; J[1] = 0.0; J[2] = -cam->fx * txc / (tz * tz);
    J[3] = 0.0; J[4] = cam->fy / tz; J[5] = -cam->fy * tyc / (tz * tz);
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int l = 0; l < 3; ++l) acc += J[3 * i + l] * R[3 * l + j];
            P->T2[3 * i + j] = acc;
        }
    double C2[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0.0;
            for (int l = 0; l < 3; ++l)
                for (int m = 0; m < 3; ++m) acc += P->T2[3 * i + l] * P->Sig[3 * l + m] * P->T2[3 * j + m];
            C2[2 * i + j] = acc;
        }
    const double dil = k->mip2d > 0.0 ? k->mip2d : k->eps2d;
    P->a = C2[0] + dil;
    P->b = C2[1];
    P->c = C2[3] + dil;
    P->det = P->a * P->c - P->b * P->b;
    if (!(P->det > 0.0)) return;
    P->comp = 1.0;
    if (k->mip2d > 0.0) {
        P->det0 = C2[0] * C2[3] - C2[1] * C2[1];
        P->comp = P->det0 > 0.0 ? sqrt(P->det0 / P->det) : 0.0;
    }
    P->conic[0] = P->c / P->det;
    P->conic[1] = -P->b / P->det;
    P->conic[2] = P->a / P->det;
    const double lam = 0.5 * (P->a + P->c) + sqrt(0.25 * (P->a - P->c) * (P->a - P->c) + P->b * P->b);
    const double r3 = 3.0 * sqrt(lam);
    P->u = cam->fx * tx / tz + cam->cx;
    P->v = cam->fy * ty / tz + cam->cy;
    /* numerical guard: degenerate footprints or centres beyond 2^30 px are culled */
    if (!(r3 <= 1073741824.0) || !(fabs(P->u) <= 1073741824.0) || !(fabs(P->v) <= 1073741824.0)) return;
    P->radius = (int64_t)ceil(r3);

    /* tile rect, floor((u -/+ r)/B) evaluated exactly as floor(floor(u) -/+ r, B) */
    const int64_t B = k->tile;
    const int64_t TX = (cam->width + B - 1) / B, TY = (cam->height + B - 1) / B;
    const int64_t fu = (int64_t)floor(P->u), fv = (int64_t)floor(P->v);
    int64_t x0 = floordiv(fu - P->radius, B), x1 = floordiv(fu + P->radius, B) + 1;
    int64_t y0 = floordiv(fv - P->radius, B), y1 = floordiv(fv + P->radius, B) + 1;
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > TX) x1 = TX;
    if (y1 > TY) y1 = TY;
    if (x0 >= x1 || y0 >= y1) return;
    P->rect[0] = x0; P->rect[1] = y0; P->rect[2] = x1; P->rect[3] = y1;

    /* view-dependent colour */
    for (int i = 0; i < 3; ++i)
        P->campos[i] = -(R[i] * cam->t[0] + R[3 + i] * cam->t[1] + R[6 + i] * cam->t[2]);
    for (int i = 0; i < 3; ++i) P->draw[i] = P->p[i] - P->campos[i];
    P->dlen = sqrt(P->draw[0] * P->draw[0] + P->draw[1] * P->draw[1] + P->draw[2] * P->draw[2]);
    for (int i = 0; i < 3; ++i) P->dir[i] = P->draw[i] / P->dlen;
    double Y[16], G[16][3];
    sh_basis(P->dir, Y, G);
    const int nb = (k->sh_degree + 1) * (k->sh_degree + 1);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int kk = 0; kk < nb; ++kk) acc += Y[kk] * g[O_SH + 3 * kk + ch];
        acc += 0.5;
        P->clamp[ch] = acc < 0.0;
        P->rgb[ch] = acc < 0.0 ? 0.0 : acc;
    }
    P->osig = 1.0 / (1.0 + exp(-g[O_OPAC]));
    P->o = P->osig * P->comp;
    P->visible = 1;
}

/* Outputs per Gaussian: feat[9] = (u, v, A, B, C, o, r, g, b), depth (t_z),
 * depth_key = bits of (float) t_z, radius (0 when culled), tiles touched,
 * rect[4] = (x0, y0, x1, y1), clamp[3]. */
void dgo_project(int64_t n, const double* g, const dgo_camera* cam, const dgo_consts* k,
                 double* feat, double* depth, uint32_t* depth_key, int32_t* radius,
                 int32_t* tiles, int32_t* rect, uint8_t* clamp)
{
    for (int64_t i = 0; i < n; ++i) {
        gproj P;
        project_one(g + NP * i, cam, k, &P);
        double* f = feat + NF * i;
        memset(f, 0, sizeof(double) * NF);
        depth[i] = P.t[2];
        float zf = (float)P.t[2];
        memcpy(&depth_key[i], &zf, 4);
        radius[i] = 0; tiles[i] = 0;
        for (int j = 0; j < 4; ++j) rect[4 * i + j] = 0;
        for (int j = 0; j < 3; ++j) clamp[3 * i + j] = 0;
        if (!P.visible) continue;
        f[0] = P.u; f[1] = P.v;
        f[2] = P.conic[0]; f[3] = P.conic[1]; f[4] = P.conic[2];
        f[5] = P.o;
        f[6] = P.rgb[0]; f[7] = P.rgb[1]; f[8] = P.rgb[2];
        radius[i] = (int32_t)P.radius;
        tiles[i] = (int32_t)((P.rect[2] - P.rect[0]) * (P.rect[3] - P.rect[1]));
        for (int j = 0; j < 4; ++j) rect[4 * i + j] = (int32_t)P.rect[j];
        for (int j = 0; j < 3; ++j) clamp[3 * i + j] = (uint8_t)P.clamp[j];
    }
}

/* ------------------------------------------------------------------ */
/* Binning: every (tile in rect, Gaussian) pair, ordered by
 * (tile id = ty*TX + tx, depth key, Gaussian index).  The rect is recomputed
 * from (u, v, radius) so that the same routine bins FP64 records and the
 * records of another implementation. */
typedef struct pair3 { uint32_t tile, key, gid; } pair3;

static int cmp_pair3(const void* pa, const void* pb)
{
    const pair3* a = (const pair3*)pa;
    const pair3* b = (const pair3*)pb;
    if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->gid != b->gid) return a->gid < b->gid ? -1 : 1;
    return 0;
}

static int rect_of(double u, double v, int64_t r, int64_t W, int64_t H, int64_t B, int64_t rc[4])
{
    const int64_t TX = (W + B - 1) / B, TY = (H + B - 1) / B;
    const int64_t fu = (int64_t)floor(u), fv = (int64_t)floor(v);
    rc[0] = floordiv(fu - r, B); rc[2] = floordiv(fu + r, B) + 1;
    rc[1] = floordiv(fv - r, B); rc[3] = floordiv(fv + r, B) + 1;
    if (rc[0] < 0) rc[0] = 0;
    if (rc[1] < 0) rc[1] = 0;
    if (rc[2] > TX) rc[2] = TX;
    if (rc[3] > TY) rc[3] = TY;
    return rc[0] < rc[2] && rc[1] < rc[3];
}

/* Returns M, the number of pairs.  Writes tile_out/gid_out/ranges only when
 * M <= capacity.  ranges has 2*TX*TY entries [start, end). */
int64_t dgo_bin(int64_t n, const double* uv, const int32_t* radius, const uint32_t* depth_key,
                int32_t W, int32_t H, int32_t B, int64_t capacity,
                uint32_t* tile_out, uint32_t* gid_out, uint32_t* ranges)
{
    const int64_t TX = (W + B - 1) / B, TY = (H + B - 1) / B;
    int64_t M = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t rc[4];
        if (radius[i] <= 0) continue;
        if (!rect_of(uv[2 * i], uv[2 * i + 1], radius[i], W, H, B, rc)) continue;
        M += (rc[2] - rc[0]) * (rc[3] - rc[1]);
    }
    if (M > capacity) return M;
    pair3* pr = (pair3*)malloc(sizeof(pair3) * (size_t)(M > 0 ? M : 1));
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t rc[4];
        if (radius[i] <= 0) continue;
        if (!rect_of(uv[2 * i], uv[2 * i + 1], radius[i], W, H, B, rc)) continue;
        for (int64_t ty = rc[1]; ty < rc[3]; ++ty)
            for (int64_t tx = rc[0]; tx < rc[2]; ++tx) {
                pr[m].tile = (uint32_t)(ty * TX + tx);
                pr[m].key = depth_key[i];
                pr[m].gid = (uint32_t)i;
                ++m;
            }
    }
    qsort(pr, (size_t)M, sizeof(pair3), cmp_pair3);
    for (int64_t t = 0; t < 2 * TX * TY; ++t) ranges[t] = 0;
    for (int64_t j = 0; j < M; ++j) {
        tile_out[j] = pr[j].tile;
        gid_out[j] = pr[j].gid;
        if (j == 0 || pr[j].tile != pr[j - 1].tile) ranges[2 * pr[j].tile] = (uint32_t)j;
        if (j == M - 1 || pr[j].tile != pr[j + 1].tile) ranges[2 * pr[j].tile + 1] = (uint32_t)(j + 1);
    }
    free(pr);
    return M;
}

/* One tile's list by the same definition, for sampled checks at full size:
 * the Gaussians whose rect contains tile `tile_id`, ordered by (depth key,
 * index).  Returns the count; writes at most `cap` indices. */
int64_t dgo_tile_list(int64_t n, const double* uv, const int32_t* radius, const uint32_t* depth_key,
                      int32_t W, int32_t H, int32_t B, int64_t tile_id, int64_t cap, uint32_t* out)
{
    const int64_t TX = (W + B - 1) / B;
    const int64_t tx = tile_id % TX, ty = tile_id / TX;
    int64_t m = 0;
    pair3* pr = NULL;
    int64_t pcap = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t rc[4];
        if (radius[i] <= 0) continue;
        if (!rect_of(uv[2 * i], uv[2 * i + 1], radius[i], W, H, B, rc)) continue;
        if (tx < rc[0] || tx >= rc[2] || ty < rc[1] || ty >= rc[3]) continue;
        if (m == pcap) {
            pcap = pcap ? 2 * pcap : 1024;
            pr = (pair3*)realloc(pr, sizeof(pair3) * (size_t)pcap);
        }
        pr[m].tile = (uint32_t)tile_id; pr[m].key = depth_key[i]; pr[m].gid = (uint32_t)i;
        ++m;
    }
    if (m > 0) qsort(pr, (size_t)m, sizeof(pair3), cmp_pair3);
    for (int64_t j = 0; j < m && j < cap; ++j) out[j] = pr[j].gid;
    free(pr);
    return m;
}

/* ------------------------------------------------------------------ */
/* Eq. 1 per pixel, front to back over the pixel's tile list. */
typedef struct blend_rec {
    uint32_t gid;
    double alpha, T, G, dx, dy;
    int clamped;
} blend_rec;

static int64_t composite_pixel(const double* feat, int32_t W, int32_t B, const uint32_t* gid,
                               const uint32_t* ranges, const dgo_consts* k, int32_t px, int32_t py,
                               double* Tout, int32_t* last_out, int32_t* examined_out,
                               double Cout[3], blend_rec* recs)
{
    const int64_t TX = (W + B - 1) / B;
    const int64_t tile = (int64_t)(py / B) * TX + (px / B);
    const uint32_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
    const double fx = px + 0.5, fy = py + 0.5;
    double T = 1.0, C[3] = {0.0, 0.0, 0.0};
    int32_t last = 0, examined = 0;
    int64_t nrec = 0;
    for (uint32_t pos = s; pos < e; ++pos) {
        ++examined;
        const double* f = feat + NF * (size_t)gid[pos];
        const double dx = f[0] - fx, dy = f[1] - fy;
        const double power = -0.5 * (f[2] * dx * dx + f[4] * dy * dy) - f[3] * dx * dy;
        if (power > 0.0) continue;
        const double G = exp(power);
        const double raw = f[5] * G;
        const int clamped = raw > k->alpha_max;
        const double alpha = clamped ? k->alpha_max : raw;
        if (alpha < k->alpha_min) continue;
        const double Tn = T * (1.0 - alpha);
        if (Tn < k->t_min) break;
        for (int ch = 0; ch < 3; ++ch) C[ch] += alpha * T * f[6 + ch];
        if (recs) {
            recs[nrec].gid = gid[pos]; recs[nrec].alpha = alpha; recs[nrec].T = T;
            recs[nrec].G = G; recs[nrec].dx = dx; recs[nrec].dy = dy; recs[nrec].clamped = clamped;
        }
        ++nrec;
        T = Tn;
        last = (int32_t)(pos - s + 1);
    }
    *Tout = T; *last_out = last; *examined_out = examined;
    for (int ch = 0; ch < 3; ++ch) Cout[ch] = C[ch];
    return nrec;
}

void dgo_render_fwd(const double* feat, int32_t W, int32_t H, int32_t B, const uint32_t* gid,
                    const uint32_t* ranges, const double* bg, const dgo_consts* k,
                    double* img, double* T_out, int32_t* last_out, int32_t* examined_out,
                    int32_t* blended_out)
{
    const int64_t HW = (int64_t)W * H;
    for (int32_t py = 0; py < H; ++py)
        for (int32_t px = 0; px < W; ++px) {
            double T, C[3];
            int32_t last, ex;
            const int64_t nb = composite_pixel(feat, W, B, gid, ranges, k, px, py, &T, &last, &ex, C, NULL);
            const int64_t i = (int64_t)py * W + px;
            for (int ch = 0; ch < 3; ++ch) img[ch * HW + i] = C[ch] + T * bg[ch];
            T_out[i] = T;
            last_out[i] = last;
            if (examined_out) examined_out[i] = ex;
            if (blended_out) blended_out[i] = (int32_t)nb;
        }
}

/* Eq. 1 at sampled pixels only (same per-pixel rule as dgo_render_fwd). */
void dgo_render_pixels(const double* feat, int32_t W, int32_t B, const uint32_t* gid, const uint32_t* ranges,
                       const double* bg, const dgo_consts* k, int64_t npix, const int32_t* px,
                       const int32_t* py, double* rgb, double* T_out, int32_t* last_out, int32_t* examined_out)
{
    for (int64_t j = 0; j < npix; ++j) {
        double T, C[3];
        int32_t last, ex;
        composite_pixel(feat, W, B, gid, ranges, k, px[j], py[j], &T, &last, &ex, C, NULL);
        for (int ch = 0; ch < 3; ++ch) rgb[3 * j + ch] = C[ch] + T * bg[ch];
        T_out[j] = T;
        last_out[j] = last;
        examined_out[j] = ex;
    }
}

/* Adjoint of Eq. 1.  grad2d (n x 9, accumulated into; caller zeroes) holds
 * dL/d(u, v, A, B, C, o, r, g, b).  dC/dc_j = alpha_j T_j;
 * dC/dalpha_j = T_j c_j - S_j / (1 - alpha_j) with S_j the colour composited
 * behind j including the background term T_N bg. */
void dgo_render_bwd(const double* feat, int32_t W, int32_t H, int32_t B, const uint32_t* gid,
                    const uint32_t* ranges, const double* bg, const dgo_consts* k,
                    const double* dL_dimg, double* grad2d)
{
    const int64_t HW = (int64_t)W * H;
    const int64_t TX = (W + B - 1) / B;
    uint32_t maxlen = 0;
    for (int64_t t = 0; t < TX * ((H + B - 1) / B); ++t)
        if (ranges[2 * t + 1] - ranges[2 * t] > maxlen) maxlen = ranges[2 * t + 1] - ranges[2 * t];
    blend_rec* recs = (blend_rec*)malloc(sizeof(blend_rec) * (maxlen + 1));
    for (int32_t py = 0; py < H; ++py)
        for (int32_t px = 0; px < W; ++px) {
            double T, C[3];
            int32_t last, ex;
            const int64_t i = (int64_t)py * W + px;
            double gpix[3];
            for (int ch = 0; ch < 3; ++ch) gpix[ch] = dL_dimg[ch * HW + i];
            if (gpix[0] == 0.0 && gpix[1] == 0.0 && gpix[2] == 0.0) continue; /* contributes exactly 0 */
            const int64_t nrec = composite_pixel(feat, W, B, gid, ranges, k, px, py, &T, &last, &ex, C, recs);
            double S[3];
            for (int ch = 0; ch < 3; ++ch) S[ch] = T * bg[ch];
            for (int64_t j = nrec - 1; j >= 0; --j) {
                const blend_rec* r = &recs[j];
                const double* f = feat + NF * (size_t)r->gid;
                double* gr = grad2d + NF * (size_t)r->gid;
                double dLda = 0.0;
                for (int ch = 0; ch < 3; ++ch) {
                    gr[6 + ch] += r->alpha * r->T * gpix[ch];
                    dLda += gpix[ch] * (r->T * f[6 + ch] - S[ch] / (1.0 - r->alpha));
                }
                for (int ch = 0; ch < 3; ++ch) S[ch] += r->alpha * r->T * f[6 + ch];
                if (r->clamped) continue;
                gr[5] += dLda * r->G;
                const double dpow = dLda * r->alpha;
                gr[0] += dpow * -(f[2] * r->dx + f[3] * r->dy);
                gr[1] += dpow * -(f[3] * r->dx + f[4] * r->dy);
                gr[2] += dpow * -0.5 * r->dx * r->dx;
                gr[3] += dpow * -r->dx * r->dy;
                gr[4] += dpow * -0.5 * r->dy * r->dy;
            }
        }
    free(recs);
}

/* ------------------------------------------------------------------ */
/* Adjoint of the projection for one Gaussian.  g2 = dL/d(u,v,A,B,C,o,r,g,b). */
static void project_bwd_one(const double* g, const dgo_camera* cam, const dgo_consts* k,
                            const double* g2, double* out)
{
    memset(out, 0, sizeof(double) * NP);
    gproj P;
    project_one(g, cam, k, &P);
    if (!P.visible) return;
    const double* R = cam->R;
    double dLdp[3] = {0.0, 0.0, 0.0};
    double dLdt[3] = {0.0, 0.0, 0.0};

    /* colour: SH coefficients and view direction */
    double dc[3];
    for (int ch = 0; ch < 3; ++ch) dc[ch] = P.clamp[ch] ? 0.0 : g2[6 + ch];
    double Y[16], G[16][3];
    sh_basis(P.dir, Y, G);
    const int nb = (k->sh_degree + 1) * (k->sh_degree + 1);
    double dLddir[3] = {0.0, 0.0, 0.0};
    for (int kk = 0; kk < nb; ++kk)
        for (int ch = 0; ch < 3; ++ch) {
            out[O_SH + 3 * kk + ch] = Y[kk] * dc[ch];
            for (int i = 0; i < 3; ++i) dLddir[i] += dc[ch] * g[O_SH + 3 * kk + ch] * G[kk][i];
        }
    const double dd = P.dir[0] * dLddir[0] + P.dir[1] * dLddir[1] + P.dir[2] * dLddir[2];
    for (int i = 0; i < 3; ++i) dLdp[i] += (dLddir[i] - P.dir[i] * dd) / P.dlen;

    /* opacity through the sigmoid (and the 2D-filter compensation) */
    out[O_OPAC] = g2[5] * P.comp * P.osig * (1.0 - P.osig);

    /* pixel mean */
    const double tx = P.t[0], ty = P.t[1], tz = P.t[2];
    dLdt[0] += g2[0] * cam->fx / tz;
    dLdt[1] += g2[1] * cam->fy / tz;
    dLdt[2] += -g2[0] * cam->fx * tx / (tz * tz) - g2[1] * cam->fy * ty / (tz * tz);

    /* conic = inverse of the 2D covariance; Gm = -K Gk K is dL/dSigma' */
    const double K[4] = {P.conic[0], P.conic[1], P.conic[1], P.conic[2]};
    const double Gk[4] = {g2[2], 0.5 * g2[3], 0.5 * g2[3], g2[4]};
    double KG[4], Gm[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) KG[2 * i + j] = K[2 * i] * Gk[j] + K[2 * i + 1] * Gk[2 + j];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) Gm[2 * i + j] = -(KG[2 * i] * K[j] + KG[2 * i + 1] * K[2 + j]);
    /* 2D filter: comp = sqrt(det0 / det), det0 of T2 Sigma T2^T, det of it plus mip2d I;
     * per matrix entry d det0 / dS00 = S11 (undilated), d det / dS00 = c (dilated), and
     * the off-diagonal entry carries half of the derivative in b */
    if (k->mip2d > 0.0 && P.det0 > 0.0) {
        const double dLdc = g2[5] * P.osig;
        const double a0 = P.a - k->mip2d, c0 = P.c - k->mip2d;
        const double h = 0.5 * P.comp * dLdc;
        Gm[0] += h * (c0 / P.det0 - P.c / P.det);
        Gm[3] += h * (a0 / P.det0 - P.a / P.det);
        Gm[1] += h * (-P.b / P.det0 + P.b / P.det);
        Gm[2] += h * (-P.b / P.det0 + P.b / P.det);
    }

    /* Sigma' = T2 Sigma T2^T + eps I:  dL/dSigma = T2^T Gm T2,  dL/dT2 = 2 Gm T2 Sigma */
    double dSig[9], dT2[6], GT[6];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int l = 0; l < 2; ++l)
                for (int m = 0; m < 2; ++m) acc += P.T2[3 * l + i] * Gm[2 * l + m] * P.T2[3 * m + j];
            dSig[3 * i + j] = acc;
        }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) GT[3 * i + j] = Gm[2 * i] * P.T2[j] + Gm[2 * i + 1] * P.T2[3 + j];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int l = 0; l < 3; ++l) acc += GT[3 * i + l] * P.Sig[3 * l + j];
            dT2[3 * i + j] = 2.0 * acc;
        }
    /* T2 = J R:  dL/dJ = dL/dT2 R^T */
    double dJ[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int l = 0; l < 3; ++l) acc += dT2[3 * i + l] * R[3 * j + l];
            dJ[3 * i + j] = acc;
        }
    /* J entries as functions of t (exact derivative of the guarded map) */
    const double fx = cam->fx, fy = cam->fy;
    dLdt[2] += dJ[0] * (-fx / (tz * tz)) + dJ[4] * (-fy / (tz * tz));
    if (!P.clampx) {
        dLdt[0] += dJ[2] * (-fx / (tz * tz));
        dLdt[2] += dJ[2] * (2.0 * fx * tx / (tz * tz * tz));
    } else {
        dLdt[2] += dJ[2] * (fx * P.limx / (tz * tz));
    }
    if (!P.clampy) {
        dLdt[1] += dJ[5] * (-fy / (tz * tz));
        dLdt[2] += dJ[5] * (2.0 * fy * ty / (tz * tz * tz));
    } else {
        dLdt[2] += dJ[5] * (fy * P.limy / (tz * tz));
    }
    /* t = R p + t_c */
    for (int i = 0; i < 3; ++i) dLdp[i] += R[i] * dLdt[0] + R[3 + i] * dLdt[1] + R[6 + i] * dLdt[2];
    for (int i = 0; i < 3; ++i) out[O_MEAN + i] = dLdp[i];

    /* Sigma = M M^T: dL/dM = 2 dL/dSigma M;  M = Rq diag(s) */
    double dM[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int l = 0; l < 3; ++l) acc += dSig[3 * i + l] * P.M[3 * l + j];
            dM[3 * i + j] = 2.0 * acc;
        }
    double dR[9];
    for (int j = 0; j < 3; ++j) {
        double ds = 0.0;
        for (int i = 0; i < 3; ++i) {
            ds += dM[3 * i + j] * P.Rq[3 * i + j];
            dR[3 * i + j] = dM[3 * i + j] * P.s[j];
        }
        out[O_LSCALE + j] = ds * P.s[j];
    }
    /* Rq(qn) */
    const double w = P.qn[0], x = P.qn[1], y = P.qn[2], z = P.qn[3];
    double dqn[4];
    dqn[0] = 2.0 * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    dqn[1] = 2.0 * (y * dR[1] + z * dR[2] + y * dR[3] - 2.0 * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] - 2.0 * x * dR[8]);
    dqn[2] = 2.0 * (-2.0 * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] - 2.0 * y * dR[8]);
    dqn[3] = 2.0 * (-2.0 * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.0 * z * dR[4] + y * dR[5] + x * dR[6] + y * dR[7]);
    /* normalisation qn = q / |q| */
    const double qd = P.qn[0] * dqn[0] + P.qn[1] * dqn[1] + P.qn[2] * dqn[2] + P.qn[3] * dqn[3];
    for (int i = 0; i < 4; ++i) out[O_QUAT + i] = (dqn[i] - P.qn[i] * qd) / P.qlen;
}

void dgo_project_bwd(int64_t n, const double* g, const dgo_camera* cam, const dgo_consts* k,
                     const double* grad2d, double* grad)
{
    for (int64_t i = 0; i < n; ++i) project_bwd_one(g + NP * i, cam, k, grad2d + NF * i, grad + NP * i);
}

/* ------------------------------------------------------------------ */
/* L1 loss, mean |img - target| over n values; grad = sign(img - target)/n
 * (zero at a tie).  Returns the loss. */
double dgo_loss_l1(int64_t n, const double* img, const double* target, double* grad)
{
    double acc = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double d = img[i] - target[i];
        acc += fabs(d);
        if (grad) grad[i] = (d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0)) / (double)n;
    }
    return acc / (double)n;
}

/* Adam (Kingma & Ba, Algorithm 1) with per-element learning rate; step >= 1. */
void dgo_adam(int64_t n, double* param, const double* grad, double* m, double* v, const double* lr,
              double beta1, double beta2, double eps, int64_t step)
{
    const double bc1 = 1.0 - pow(beta1, (double)step);
    const double bc2 = 1.0 - pow(beta2, (double)step);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
        const double mh = m[i] / bc1, vh = v[i] / bc2;
        param[i] -= lr[i] * mh / (sqrt(vh) + eps);
    }
}
