/*
 * Seeded procedural scene generator: analytic spheres resting on a ground plane, seen by a
 * pinhole camera that pans (yaw) by a fixed screen distance per frame, lit by one point light
 * with hard shadows.  Per frame it writes
 *   - noisy radiance   : noise-free radiance x an Exp(1) factor per pixel (a 1-spp stand-in;
 *                        with rough_noise the factor is 1 + r (Exp(1) - 1), r the surface
 *                        roughness, so smooth surfaces are less noisy), clamped to
 *                        [0, max_radiance]                                   float [H][W][3]
 *   - noise-free radiance (ground truth, same clamp)                        float [H][W][3]
 *   - G-buffer         : world-space unit normal + linear (view-axis) depth float [H][W][4]
 *   - screen motion    : mv = p_cur - p_prev in pixels (pixel-centre convention) [H][W][2]
 *   - roughness        : per object, never within 0.01 of 0.2 (or one value for every
 *                        surface)                                          float [H][W]
 *   - albedo           : per object, U[0.1, 0.9] per channel               float [H][W][3]
 * and, from scene_render_shadow, a shadow channel for a spherical light of radius light_radius
 * at the point light's position:
 *   - shadow_noisy     : visibility of one uniform sample on the light's disk (0 or 1)
 *   - shadow_gt        : visibility fraction over 8 x 8 stratified disk samples
 *   - shadow_angle     : the light's angular diameter seen from the surface, in degrees
 * With moving_light the light circles (radius 3, 0.05 rad per frame) above its start position.
 *
 * This is input infrastructure shared by the CUDA path's tests and benchmark and by the CPU
 * oracle's tests. It holds none of the denoiser's arithmetic. Everything is computed in FP64
 * and rounded to FP32 on output. Random numbers come from SplitMix64 (Steele, Lea & Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014): the scene layout from a
 * sequential SplitMix64 stream, the per-pixel noise from its finaliser applied to a counter
 * (seed, stream, frame, pixel), so any frame can be generated on its own.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int width, height;
    int n_spheres;
    int moving_sphere;          /* 1: sphere 0 moves across the view (disocclusions) */
    double pan_px_per_frame;    /* camera yaw per frame, as pixels at the image centre */
    double moving_px_per_frame; /* screen speed of the moving sphere */
    double vfov_deg;            /* vertical field of view */
    double max_radiance;        /* HDR clamp */
    uint64_t seed;
    uint64_t stream;
    double roughness;           /* < 0: drawn per object; otherwise every surface's roughness */
    int rough_noise;            /* 1: noise factor 1 + roughness (Exp(1) - 1) */
    int moving_light;           /* 1: the light circles over the scene */
    double light_radius;        /* radius of the spherical light of the shadow channel */
} scene_config;

#define MAX_SPHERES 256

typedef struct { double x, y, z; } v3;
static v3 v3_make(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return v3_make(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return v3_make(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return v3_make(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) {
    return v3_make(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static v3 normalize(v3 a) { return scl(a, 1.0 / sqrt(dot(a, a))); }

/* SplitMix64 finaliser and sequential generator. */
static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static uint64_t sm_next(uint64_t* s) {
    *s += 0x9E3779B97F4A7C15ull;
    return mix64(*s);
}
static double unit_double(uint64_t z) { return (double)(z >> 11) * (1.0 / 9007199254740992.0); }
static double sm_uniform(uint64_t* s, double lo, double hi) {
    return lo + (hi - lo) * unit_double(sm_next(s));
}

typedef struct {
    v3 c0;            /* centre at frame 0 */
    double r;
    v3 albedo;
    double roughness;
} sphere;

typedef struct {
    int n;
    sphere s[MAX_SPHERES];
    v3 plane_albedo;
    double plane_roughness;
    v3 light;
    double light_intensity;
    double ambient;
    v3 cam_pos;
    double pitch;     /* radians, looking down */
    double f_px;      /* focal length in pixels */
    double yaw_step;  /* radians per frame */
    v3 velocity;      /* world displacement per frame of sphere 0 when moving */
} scene;

/* Roughness per object, kept away from the 0.2 adaptive-start threshold so that no pixel's
 * decision sits on it. */
static double draw_roughness(uint64_t* s) {
    for (;;) {
        double r = sm_uniform(s, 0.0, 1.0);
        if (fabs(r - 0.2) >= 0.01) return r;
    }
}

typedef struct { v3 f, r, u; } cam_basis;

static cam_basis camera_at(const scene* sc, int frame) {
    double th = sc->yaw_step * (double)frame, ph = sc->pitch;
    cam_basis b;
    b.f = v3_make(sin(th) * cos(ph), -sin(ph), cos(th) * cos(ph));
    b.r = v3_make(cos(th), 0.0, -sin(th));
    b.u = cross(b.f, b.r);
    return b;
}

static void build_scene(const scene_config* cfg, scene* sc) {
    uint64_t st = mix64(cfg->seed * 0xD1B54A32D192ED03ull + 0x8CB92BA72F3D8DD7ull) ^
                  mix64(cfg->stream + 0x632BE59BD9B4E019ull);
    double W = cfg->width, H = cfg->height;
    sc->n = cfg->n_spheres < MAX_SPHERES ? cfg->n_spheres : MAX_SPHERES;
    sc->cam_pos = v3_make(0.0, 3.0, -6.0);
    sc->pitch = 30.0 * M_PI / 180.0;
    sc->f_px = 0.5 * H / tan(0.5 * cfg->vfov_deg * M_PI / 180.0);
    sc->yaw_step = atan(cfg->pan_px_per_frame / sc->f_px);
    sc->plane_albedo = v3_make(sm_uniform(&st, 0.1, 0.9), sm_uniform(&st, 0.1, 0.9),
                               sm_uniform(&st, 0.1, 0.9));
    sc->plane_roughness = draw_roughness(&st);
    if (cfg->roughness >= 0.0) sc->plane_roughness = cfg->roughness;
    sc->light = v3_make(4.0, 12.0, 2.0);
    sc->light_intensity = 400.0;
    sc->ambient = 0.05;
    for (int i = 0; i < sc->n; ++i) {
        sphere* s = &sc->s[i];
        s->r = sm_uniform(&st, 0.4, 1.5);
        double x = sm_uniform(&st, -8.0, 8.0), z = sm_uniform(&st, 3.0, 22.0);
        s->c0 = v3_make(x, s->r, z);
        s->albedo = v3_make(sm_uniform(&st, 0.1, 0.9), sm_uniform(&st, 0.1, 0.9),
                            sm_uniform(&st, 0.1, 0.9));
        s->roughness = draw_roughness(&st);
        if (cfg->roughness >= 0.0) s->roughness = cfg->roughness;
    }
    sc->velocity = v3_make(0.0, 0.0, 0.0);
    if (cfg->moving_sphere && sc->n > 0) {
        /* Sphere 0: radius 1, on the plane, 10 units down the frame-0 view axis and a quarter
         * of the image width left of centre; it moves along the frame-0 right axis. */
        cam_basis b = camera_at(sc, 0);
        v3 fh = normalize(v3_make(b.f.x, 0.0, b.f.z));
        double depth = 10.0;
        v3 c = add(sc->cam_pos, scl(fh, depth));
        c = add(c, scl(b.r, -0.25 * W * depth / sc->f_px));
        c.y = 1.0;
        sc->s[0].r = 1.0;
        sc->s[0].c0 = c;
        double zc = dot(sub(c, sc->cam_pos), b.f);
        sc->velocity = scl(b.r, cfg->moving_px_per_frame * zc / sc->f_px);
    }
}

static v3 light_at(const scene* sc, const scene_config* cfg, int frame) {
    if (!cfg->moving_light) return sc->light;
    double a = 0.05 * (double)frame;
    return add(sc->light, v3_make(3.0 * cos(a) - 3.0, 0.0, 3.0 * sin(a)));
}

static v3 sphere_centre(const scene* sc, int i, int frame) {
    v3 c = sc->s[i].c0;
    if (i == 0) c = add(c, scl(sc->velocity, (double)frame));
    return c;
}

/* Nearest positive root of |o + t d - c|^2 = r^2 (d unit), or -1. */
static double hit_sphere(v3 o, v3 d, v3 c, double r) {
    v3 oc = sub(o, c);
    double b = dot(oc, d), cc = dot(oc, oc) - r * r;
    double disc = b * b - cc;
    if (disc < 0.0) return -1.0;
    double sq = sqrt(disc);
    double t = -b - sq;
    if (t > 1e-9) return t;
    t = -b + sq;
    return t > 1e-9 ? t : -1.0;
}

/* 64-bit key of one pixel's noise draw. */
static uint64_t pixel_key(uint64_t seed, uint64_t stream, uint64_t frame, uint64_t pixel) {
    uint64_t k = mix64(seed + 0x9E3779B97F4A7C15ull);
    k = mix64(k ^ (stream + 0x3C6EF372FE94F82Aull));
    k = mix64(k ^ (frame + 0xDAA66D2C7DDF743Full));
    return mix64(k ^ (pixel + 0x78DDE6E5FD29F054ull));
}

/* The camera ray through pixel (x, y): hit point P, normal N, albedo, roughness, object
 * (-1 plane, >= 0 sphere index, -2 nothing). */
typedef struct { v3 P, N, alb; double rough; int obj; } surface;

static surface primary_hit(const scene* sc, const v3* centres, cam_basis cb, int W, int H, int x,
                           int y) {
    double px = x + 0.5, py = y + 0.5;
    v3 d = add(cb.f, add(scl(cb.r, (px - 0.5 * W) / sc->f_px), scl(cb.u, -(py - 0.5 * H) / sc->f_px)));
    d = normalize(d);
    v3 o = sc->cam_pos;
    double tbest = 1e300;
    surface s;
    s.obj = -2;
    if (d.y < 0.0) {
        double t = -o.y / d.y;
        if (t > 1e-9) { tbest = t; s.obj = -1; }
    }
    for (int i = 0; i < sc->n; ++i) {
        double t = hit_sphere(o, d, centres[i], sc->s[i].r);
        if (t > 0.0 && t < tbest) { tbest = t; s.obj = i; }
    }
    if (s.obj == -2) {
        /* Not reached with the fixed 30 degree pitch; kept well defined anyway. */
        tbest = 1e4;
        s.P = add(o, scl(d, tbest));
        s.N = scl(cb.f, -1.0);
        s.alb = v3_make(0.0, 0.0, 0.0);
        s.rough = 1.0;
    } else {
        s.P = add(o, scl(d, tbest));
        if (s.obj == -1) {
            s.N = v3_make(0.0, 1.0, 0.0);
            s.alb = sc->plane_albedo;
            s.rough = sc->plane_roughness;
        } else {
            s.N = normalize(sub(s.P, centres[s.obj]));
            s.alb = sc->s[s.obj].albedo;
            s.rough = sc->s[s.obj].roughness;
        }
    }
    return s;
}

/* 1 if the segment from the surface point (offset along N) to Q is not blocked by a sphere. */
static double visible(const scene* sc, const v3* centres, v3 P, v3 N, v3 Q) {
    v3 L = sub(Q, P);
    double dl = sqrt(dot(L, L));
    v3 l = scl(L, 1.0 / dl);
    if (dot(N, l) <= 0.0) return 0.0;
    v3 so = add(P, scl(N, 1e-4));
    for (int i = 0; i < sc->n; ++i) {
        double t = hit_sphere(so, l, centres[i], sc->s[i].r);
        if (t > 0.0 && t < dl) return 0.0;
    }
    return 1.0;
}

int scene_render_frame(const scene_config* cfg, int frame, float* noisy, float* gt,
                       float* gbuf_nz, float* motion, float* roughness, float* albedo) {
    if (!cfg || cfg->width <= 0 || cfg->height <= 0 || cfg->n_spheres < 0) return 1;
    scene sc;
    build_scene(cfg, &sc);
    const int W = cfg->width, H = cfg->height;
    cam_basis cb = camera_at(&sc, frame), pb = camera_at(&sc, frame - 1);
    v3 centres[MAX_SPHERES];
    for (int i = 0; i < sc.n; ++i) centres[i] = sphere_centre(&sc, i, frame);
    const double maxr = cfg->max_radiance;
    const v3 light = light_at(&sc, cfg, frame);

#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            double px = x + 0.5, py = y + 0.5;
            const v3 o = sc.cam_pos;
            surface sf = primary_hit(&sc, centres, cb, W, H, x, y);
            const int obj = sf.obj;
            const v3 P = sf.P, N = sf.N, alb = sf.alb;
            const double rough = sf.rough;
            /* Lambert + point light with a hard shadow, plus a small ambient term. */
            v3 L = sub(light, P);
            double d2 = dot(L, L), dl = sqrt(d2);
            v3 l = scl(L, 1.0 / dl);
            double cosv = dot(N, l);
            double vis = cosv > 0.0 ? 1.0 : 0.0;
            if (vis > 0.0) {
                v3 so = add(P, scl(N, 1e-4));
                for (int i = 0; i < sc.n; ++i) {
                    double t = hit_sphere(so, l, centres[i], sc.s[i].r);
                    if (t > 0.0 && t < dl) { vis = 0.0; break; }
                }
            }
            double direct = obj == -2 ? 0.0 : sc.light_intensity * (cosv > 0 ? cosv : 0.0) * vis / d2;
            double rad[3] = {alb.x * (sc.ambient + direct), alb.y * (sc.ambient + direct),
                             alb.z * (sc.ambient + direct)};
            double u = unit_double(pixel_key(cfg->seed, cfg->stream, (uint64_t)(int64_t)frame, p));
            double e = -log1p(-u); /* Exp(1) */
            if (cfg->rough_noise) e = 1.0 + rough * (e - 1.0);
            for (int c = 0; c < 3; ++c) {
                double g = rad[c] < maxr ? rad[c] : maxr;
                double nz = rad[c] * e;
                nz = nz < maxr ? nz : maxr;
                if (gt) gt[3 * p + c] = (float)g;
                if (noisy) noisy[3 * p + c] = (float)nz;
                if (albedo) albedo[3 * p + c] = (float)(c == 0 ? alb.x : c == 1 ? alb.y : alb.z);
            }
            if (gbuf_nz) {
                gbuf_nz[4 * p + 0] = (float)N.x;
                gbuf_nz[4 * p + 1] = (float)N.y;
                gbuf_nz[4 * p + 2] = (float)N.z;
                gbuf_nz[4 * p + 3] = (float)dot(sub(P, o), cb.f);
            }
            if (roughness) roughness[p] = (float)rough;
            if (motion) {
                v3 Pp = P;
                if (obj == 0) Pp = sub(P, sc.velocity);
                v3 rel = sub(Pp, o);
                double zc = dot(rel, pb.f);
                double sx = 0.5 * W + sc.f_px * dot(rel, pb.r) / zc;
                double sy = 0.5 * H - sc.f_px * dot(rel, pb.u) / zc;
                motion[2 * p + 0] = (float)(px - sx);
                motion[2 * p + 1] = (float)(py - sy);
            }
        }
    }
    return 0;
}

/* Shadow channel of the spherical light (radius light_radius, centre at the point light): per
 * pixel the visibility of one uniform sample on the light's disk facing the surface point (the
 * 1-spp estimate), the 8 x 8 stratified estimate, and the light's angular diameter in degrees.
 * The disk sample of pixel p uses the SplitMix64 finaliser of (seed, stream, frame, p) with a
 * key distinct from the radiance noise. */
int scene_render_shadow(const scene_config* cfg, int frame, float* shadow_noisy, float* shadow_gt,
                        float* shadow_angle) {
    if (!cfg || cfg->width <= 0 || cfg->height <= 0 || cfg->n_spheres < 0 ||
        !(cfg->light_radius > 0.0))
        return 1;
    scene sc;
    build_scene(cfg, &sc);
    const int W = cfg->width, H = cfg->height;
    cam_basis cb = camera_at(&sc, frame);
    v3 centres[MAX_SPHERES];
    for (int i = 0; i < sc.n; ++i) centres[i] = sphere_centre(&sc, i, frame);
    const v3 light = light_at(&sc, cfg, frame);
    const double R = cfg->light_radius;

#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            surface sf = primary_hit(&sc, centres, cb, W, H, x, y);
            v3 L = sub(light, sf.P);
            double dl = sqrt(dot(L, L));
            v3 l = scl(L, 1.0 / dl);
            /* orthonormal basis (t, b) of the disk facing the surface point */
            v3 a = fabs(l.y) < 0.9 ? v3_make(0.0, 1.0, 0.0) : v3_make(1.0, 0.0, 0.0);
            v3 t = normalize(cross(a, l)), b = cross(l, t);
            if (shadow_noisy) {
                uint64_t k = pixel_key(cfg->seed ^ 0x5DEECE66Dull, cfg->stream, (uint64_t)(int64_t)frame, p);
                double u1 = unit_double(k), u2 = unit_double(mix64(k + 0x9E3779B97F4A7C15ull));
                double rr = R * sqrt(u1), ph = 2.0 * M_PI * u2;
                v3 Q = add(light, add(scl(t, rr * cos(ph)), scl(b, rr * sin(ph))));
                shadow_noisy[p] = sf.obj == -2 ? 0.0f : (float)visible(&sc, centres, sf.P, sf.N, Q);
            }
            if (shadow_gt) {
                double v = 0.0;
                for (int i = 0; i < 8; ++i)
                    for (int j = 0; j < 8; ++j) {
                        double rr = R * sqrt((i + 0.5) / 8.0), ph = 2.0 * M_PI * (j + 0.5) / 8.0;
                        v3 Q = add(light, add(scl(t, rr * cos(ph)), scl(b, rr * sin(ph))));
                        v += visible(&sc, centres, sf.P, sf.N, Q);
                    }
                shadow_gt[p] = sf.obj == -2 ? 0.0f : (float)(v / 64.0);
            }
            if (shadow_angle) shadow_angle[p] = (float)(2.0 * asin(R < dl ? R / dl : 1.0) * 180.0 / M_PI);
        }
    }
    return 0;
}
