// Host-side check of the halo-free 3D tiling (no GPU call): for every grid the
// halo-free kernels accept and every CTA cap and CTAs-per-SM setting, the
// tiling returned by the library covers the grid exactly, fits the reduction
// scratch and the shared memory of the kernels, and reports the face-buffer
// size it indexes.  Prints one line per violation and "ok <cases>" at the end.
#include <cstdio>

#include "stencil_v2.cuh"

using namespace jfnk;

static long long fixup_count(const V2Geom& q) {
    const long long m1 = q.n - 1;
    return (long long)(q.Ty - 1) * m1 * m1 + (long long)(q.Tz - 1) * (m1 - (q.Ty - 1)) * m1;
}

int main() {
    int bad = 0, cases = 0;
    for (int n = 64; n <= 512; n += 32) {
        const Grid g = Grid::make(3, n);
        if (!v2_applicable(g)) {
            printf("n=%d: not applicable\n", n);
            ++bad;
            continue;
        }
        for (int cap : {1024, 512, 256}) {
            for (int ctas : {1, 2}) {
                ++cases;
                const V2Geom q = v2_geometry(g, ctas * kNumSMs, cap);
                const long long fb = std::min<long long>(std::max<long long>((fixup_count(q) + 255) / 256, 1),
                                                         4LL * kNumSMs);
                const long long ysz = (long long)q.Ty * q.Tz * (q.ZC + 1) * (n + 1);
                const long long zsz = (long long)q.Ty * q.Tz * (q.BY + 1) * (n + 1);
                const size_t v3_smem = sizeof(float) * (3 * (size_t)(q.BY + 1) * (n + 2) + 16 * (size_t)q.BY * (n + 2));
                // the cap holds where it can (a row of n threads is the smallest CTA)
                const bool ok_tiles = q.n == n && q.BY >= 1 && n % q.BY == 0 && q.Ty * q.BY == n &&
                                      (long long)n * q.BY <= std::max(cap, n) && n * q.BY <= kV2Threads;
                const bool ok_chunks = q.Tz >= 1 && (long long)(q.Tz - 1) * q.ZC < n && (long long)q.Tz * q.ZC >= n;
                const bool ok_faces = q.face_count == 2 * ysz + 2 * zsz && q.ylo == 0 && q.yhi == ysz &&
                                      q.zlo == 2 * ysz && q.zhi == 2 * ysz + zsz &&
                                      v3_face_count(g, cap, ctas) == q.face_count;
                // the paired variant's CTA and shared memory (2 CTAs per SM: half the opt-in limit)
                const bool ok_v3 = (n / 2) * q.BY <= kV3Threads && v3_smem <= (size_t)220 * 1024 / ctas;
                // launches with more partials than the scratch holds are refused by the launcher;
                // the tiling must keep every accepted size within it
                const bool ok_red = (long long)q.Ty * q.Tz + fb <= 2LL * kMaxRedBlocks;
                if (!(ok_tiles && ok_chunks && ok_faces && ok_v3 && ok_red)) {
                    printf("n=%d cap=%d ctas=%d: BY=%d Ty=%d Tz=%d ZC=%d tiles=%d chunks=%d faces=%d v3=%d red=%d\n", n,
                           cap, ctas, q.BY, q.Ty, q.Tz, q.ZC, ok_tiles, ok_chunks, ok_faces, ok_v3, ok_red);
                    ++bad;
                }
            }
        }
    }
    if (bad == 0) printf("ok %d\n", cases);
    return bad == 0 ? 0 : 1;
}
