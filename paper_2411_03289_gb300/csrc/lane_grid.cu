// Candidate lists for the distance to the lane polyline (Eq. 11, 13-14).
//
// The rollout needs, for every sample and stage, the distance from the mean
// position to the nearest segment of the lane's centre polyline.  Scanning all
// segments costs O(S) per sample-step; this grid makes it O(candidates).  The
// bounding box of the path, widened by a margin, is cut into square cells.
// For cell C let U_C = min_s max_{p in C} d(p, s) (the distance function of a
// segment is convex, so the inner max is attained at a corner of C).  Every
// point of C then has some segment within U_C, so a segment s with
// d(C, s) > U_C (the distance between the cell rectangle and s) can never be
// the nearest one for a point of C: the candidate list of C holds the segments
// with d(C, s) <= U_C + slack, and the minimum over the candidates equals the
// minimum over all segments.  Points outside the grid scan every segment.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace gpm {
namespace {

struct Seg {
    double ax, ay, bx, by;
};

double point_seg(double px, double py, const Seg& s) {
    const double dx = s.bx - s.ax, dy = s.by - s.ay;
    const double l2 = dx * dx + dy * dy;
    double t = l2 > 0.0 ? ((px - s.ax) * dx + (py - s.ay) * dy) / l2 : 0.0;
    t = std::min(1.0, std::max(0.0, t));
    return std::hypot(px - s.ax - t * dx, py - s.ay - t * dy);
}

double point_rect(double px, double py, double x0, double y0, double x1, double y1) {
    const double dx = std::max({x0 - px, 0.0, px - x1});
    const double dy = std::max({y0 - py, 0.0, py - y1});
    return std::hypot(dx, dy);
}

// whether the segment meets the closed rectangle (Liang-Barsky clipping)
bool seg_meets_rect(const Seg& s, double x0, double y0, double x1, double y1) {
    double t0 = 0.0, t1 = 1.0;
    const double dx = s.bx - s.ax, dy = s.by - s.ay;
    const double p[4] = {-dx, dx, -dy, dy};
    const double q[4] = {s.ax - x0, x1 - s.ax, s.ay - y0, y1 - s.ay};
    for (int i = 0; i < 4; ++i) {
        if (p[i] == 0.0) {
            if (q[i] < 0.0) return false;
        } else {
            const double r = q[i] / p[i];
            if (p[i] < 0.0) t0 = std::max(t0, r);
            else t1 = std::min(t1, r);
            if (t0 > t1) return false;
        }
    }
    return true;
}

// distance between a segment and a rectangle (0 when they meet): for two
// disjoint convex polygons it is attained at a vertex of one of them
double rect_seg(const Seg& s, double x0, double y0, double x1, double y1) {
    if (seg_meets_rect(s, x0, y0, x1, y1)) return 0.0;
    double d = std::min(point_rect(s.ax, s.ay, x0, y0, x1, y1), point_rect(s.bx, s.by, x0, y0, x1, y1));
    d = std::min(d, point_seg(x0, y0, s));
    d = std::min(d, point_seg(x1, y0, s));
    d = std::min(d, point_seg(x0, y1, s));
    d = std::min(d, point_seg(x1, y1, s));
    return d;
}

}  // namespace

int build_lane_grid(const float* path, int P, LaneGridHost& g) {
    g = LaneGridHost{};
    if (P < 2) return GPMPPI_OK;            // a single point: nothing to accelerate
    std::vector<Seg> segs(P - 1);
    double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
    for (int i = 0; i < P; ++i) {
        xmin = std::min(xmin, (double)path[2 * i]);
        xmax = std::max(xmax, (double)path[2 * i]);
        ymin = std::min(ymin, (double)path[2 * i + 1]);
        ymax = std::max(ymax, (double)path[2 * i + 1]);
    }
    for (int i = 0; i + 1 < P; ++i)
        segs[i] = Seg{path[2 * i], path[2 * i + 1], path[2 * i + 2], path[2 * i + 3]};
    const double margin = 3.0;              // metres around the path covered by the grid
    xmin -= margin;
    ymin -= margin;
    xmax += margin;
    ymax += margin;
    // about 4096 square cells over the box
    double h = std::sqrt((xmax - xmin) * (ymax - ymin) / 4096.0);
    h = std::max(h, 0.05);
    const int nx = std::min(1024, (int)std::ceil((xmax - xmin) / h));
    const int ny = std::min(1024, (int)std::ceil((ymax - ymin) / h));
    h = std::max((xmax - xmin) / nx, (ymax - ymin) / ny);
    const double slack = 1e-3;              // covers FP32 rounding of the distances on the device
    g.x0 = (float)xmin;
    g.y0 = (float)ymin;
    g.inv_h = (float)(1.0 / h);
    g.nx = nx;
    g.ny = ny;
    g.cells.resize((size_t)nx * ny);
    const int ns = (int)segs.size();
    std::vector<double> dc(ns);
    for (int iy = 0; iy < ny; ++iy)
        for (int ix = 0; ix < nx; ++ix) {
            // the cell as the device sees it: [x0 + ix h, x0 + (ix+1) h), widened by
            // the float rounding of the index computation
            const double eps = 1e-4 * h;
            const double cx0 = xmin + ix * h - eps, cx1 = xmin + (ix + 1) * h + eps;
            const double cy0 = ymin + iy * h - eps, cy1 = ymin + (iy + 1) * h + eps;
            const double mx = 0.5 * (cx0 + cx1), my = 0.5 * (cy0 + cy1);
            const double r = 0.5 * std::hypot(cx1 - cx0, cy1 - cy0);    // centre to corner
            // d(centre, s) <= max over the corners of d(corner, s) <= d(centre, s) + r
            // (convexity and the triangle inequality), so only segments with
            // d(centre, s) <= min_s d(centre, s) + r can attain U_C, and a segment
            // with d(centre, s) - r > U_C is farther than U_C from the whole cell
            double dmin = INFINITY;
            for (int i = 0; i < ns; ++i) {
                dc[i] = point_seg(mx, my, segs[i]);
                dmin = std::min(dmin, dc[i]);
            }
            double U = INFINITY;
            for (int i = 0; i < ns; ++i) {
                if (dc[i] > dmin + r) continue;
                const Seg& s = segs[i];
                const double m = std::max({point_seg(cx0, cy0, s), point_seg(cx1, cy0, s), point_seg(cx0, cy1, s),
                                           point_seg(cx1, cy1, s)});
                U = std::min(U, m);
            }
            const int off = (int)g.idx.size();
            for (int i = 0; i < ns; ++i) {
                if (dc[i] - r > U + slack) continue;
                if (rect_seg(segs[i], cx0, cy0, cx1, cy1) <= U + slack) g.idx.push_back(i);
            }
            g.cells[(size_t)iy * nx + ix] = make_int2(off, (int)g.idx.size() - off);
        }
    return GPMPPI_OK;
}

}  // namespace gpm
