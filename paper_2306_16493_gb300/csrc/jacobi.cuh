// Cyclic two-sided Jacobi eigensolver for small complex Hermitian matrices, FP64.
//
// For each off-diagonal element a_pq = |a_pq| e^{i phi} the unitary plane rotation
// U = [[c, s e^{i phi}], [-s e^{-i phi}, c]] (rows/columns p, q) zeroes it: writing
// A = D B D^dag with D = diag(1, e^{-i phi}) and B the real symmetric 2x2 block
// [[a_pp, |a_pq|], [|a_pq|, a_qq]], U = D J D^dag with the classical real rotation
// J = [[c, s], [-s, c]], t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// zeta = (a_qq - a_pp) / (2 |a_pq|), c = 1/sqrt(1 + t^2), s = t c (Golub & Van Loan,
// Matrix Computations, Sec. 8.5), so U^dag A U is diagonal in the (p, q) block.
// Sweeps repeat until the off-diagonal Frobenius norm is below 1e-15 of the full norm.
// Eigenvalues are returned ascending with the eigenvector columns of V permuted alike.
// Accurate for near-degenerate bands and soft modes (each rotation is backward stable).
#pragma once

template <int NMAX>
__host__ __device__ inline int jacobi_hermitian(double2 (&A)[NMAX * NMAX], double2 (&V)[NMAX * NMAX],
                                                int n, double *w) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[i * n + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    int converged = 0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0, tot = 0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double m2 = A[i * n + j].x * A[i * n + j].x + A[i * n + j].y * A[i * n + j].y;
                tot += m2;
                if (i != j) off += m2;
            }
        if (off <= 1e-30 * tot || off == 0.0) {
            converged = 1;
            break;
        }
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                const double2 apq = A[p * n + q];
                const double mag = sqrt(apq.x * apq.x + apq.y * apq.y);
                if (mag == 0.0) continue;
                const double app = A[p * n + p].x, aqq = A[q * n + q].x;
                const double zeta = (aqq - app) / (2.0 * mag);
                double t;
                if (fabs(zeta) > 1e150) t = 0.5 / zeta;
                else t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t);
                const double s = t * c;
                const double2 e = make_double2(apq.x / mag, apq.y / mag);          // e^{i phi}
                const double2 se = make_double2(s * e.x, s * e.y);                  // s e^{i phi}
                const double2 sec = make_double2(s * e.x, -s * e.y);                // s e^{-i phi}
                // columns: A <- A U, V <- V U
                for (int r = 0; r < n; ++r) {
                    const double2 ap = A[r * n + p], aq = A[r * n + q];
                    // A_rp c + A_rq (-s e^{-i phi});  A_rp s e^{i phi} + A_rq c
                    A[r * n + p] = make_double2(c * ap.x - (sec.x * aq.x - sec.y * aq.y),
                                                c * ap.y - (sec.x * aq.y + sec.y * aq.x));
                    A[r * n + q] = make_double2(se.x * ap.x - se.y * ap.y + c * aq.x,
                                                se.x * ap.y + se.y * ap.x + c * aq.y);
                    const double2 vp = V[r * n + p], vq = V[r * n + q];
                    V[r * n + p] = make_double2(c * vp.x - (sec.x * vq.x - sec.y * vq.y),
                                                c * vp.y - (sec.x * vq.y + sec.y * vq.x));
                    V[r * n + q] = make_double2(se.x * vp.x - se.y * vp.y + c * vq.x,
                                                se.x * vp.y + se.y * vp.x + c * vq.y);
                }
                // rows: A <- U^dag A
                for (int col = 0; col < n; ++col) {
                    const double2 bp = A[p * n + col], bq = A[q * n + col];
                    // c B_p - s e^{i phi} B_q;  s e^{-i phi} B_p + c B_q
                    A[p * n + col] = make_double2(c * bp.x - (se.x * bq.x - se.y * bq.y),
                                                  c * bp.y - (se.x * bq.y + se.y * bq.x));
                    A[q * n + col] = make_double2(sec.x * bp.x - sec.y * bp.y + c * bq.x,
                                                  sec.x * bp.y + sec.y * bp.x + c * bq.y);
                }
                A[p * n + q] = make_double2(0, 0);
                A[q * n + p] = make_double2(0, 0);
                A[p * n + p] = make_double2(app - t * mag, 0);
                A[q * n + q] = make_double2(aqq + t * mag, 0);
            }
        }
    }
    for (int i = 0; i < n; ++i) w[i] = A[i * n + i].x;
    // selection sort, ascending, permuting the eigenvector columns
    for (int i = 0; i < n - 1; ++i) {
        int k = i;
        for (int j = i + 1; j < n; ++j)
            if (w[j] < w[k]) k = j;
        if (k != i) {
            const double tw = w[i];
            w[i] = w[k];
            w[k] = tw;
            for (int r = 0; r < n; ++r) {
                const double2 tv = V[r * n + i];
                V[r * n + i] = V[r * n + k];
                V[r * n + k] = tv;
            }
        }
    }
    return converged;
}

// Mixed-precision variant with the same FP64 result (GB300 runs FP64 at 1/64 of the FP32
// rate): (1) the rotations of jacobi_hermitian in FP32 on a rounded copy of A, until the
// off-diagonal norm is below ~3e-6 of the full norm (FP32 cannot go much further) or 30 sweeps;
// (2) those eigenvectors made orthonormal in FP64 (one modified Gram-Schmidt pass, starting
// from columns orthonormal to FP32 accuracy); (3) B = V1^dag A V1 in FP64, diagonal to FP32
// accuracy; (4) jacobi_hermitian on B in FP64, which converges in one or two sweeps and
// handles (near-)degenerate blocks like the plain solver; (5) V = V1 Q.  The stopping rule of
// the FP64 stage is that of jacobi_hermitian, so the eigenpairs are FP64-accurate.
template <int NMAX>
__host__ __device__ inline int jacobi_hermitian_mixed(double2 (&A)[NMAX * NMAX], double2 (&V)[NMAX * NMAX],
                                                      int n, double *w) {
    float2 a[NMAX * NMAX], v[NMAX * NMAX];
    for (int i = 0; i < n * n; ++i) a[i] = make_float2((float)A[i].x, (float)A[i].y);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) v[i * n + j] = make_float2(i == j ? 1.f : 0.f, 0.f);
    for (int sweep = 0; sweep < 30; ++sweep) {
        float off = 0, tot = 0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const float m2 = a[i * n + j].x * a[i * n + j].x + a[i * n + j].y * a[i * n + j].y;
                tot += m2;
                if (i != j) off += m2;
            }
        if (off <= 1e-11f * tot) break;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                const float2 apq = a[p * n + q];
                const float mag = sqrtf(apq.x * apq.x + apq.y * apq.y);
                if (mag == 0.f) continue;
                const float app = a[p * n + p].x, aqq = a[q * n + q].x;
                const float zeta = (aqq - app) / (2.f * mag);
                const float t = fabsf(zeta) > 1e18f ? 0.5f / zeta
                                                    : (zeta >= 0 ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
                const float c = 1.f / sqrtf(1.f + t * t), sn = t * c;
                const float2 e = make_float2(apq.x / mag, apq.y / mag);
                const float2 se = make_float2(sn * e.x, sn * e.y), sec = make_float2(sn * e.x, -sn * e.y);
                for (int r = 0; r < n; ++r) {
                    const float2 ap = a[r * n + p], aq = a[r * n + q];
                    a[r * n + p] = make_float2(c * ap.x - (sec.x * aq.x - sec.y * aq.y), c * ap.y - (sec.x * aq.y + sec.y * aq.x));
                    a[r * n + q] = make_float2(se.x * ap.x - se.y * ap.y + c * aq.x, se.x * ap.y + se.y * ap.x + c * aq.y);
                    const float2 vp = v[r * n + p], vq = v[r * n + q];
                    v[r * n + p] = make_float2(c * vp.x - (sec.x * vq.x - sec.y * vq.y), c * vp.y - (sec.x * vq.y + sec.y * vq.x));
                    v[r * n + q] = make_float2(se.x * vp.x - se.y * vp.y + c * vq.x, se.x * vp.y + se.y * vp.x + c * vq.y);
                }
                for (int col = 0; col < n; ++col) {
                    const float2 bp = a[p * n + col], bq = a[q * n + col];
                    a[p * n + col] = make_float2(c * bp.x - (se.x * bq.x - se.y * bq.y), c * bp.y - (se.x * bq.y + se.y * bq.x));
                    a[q * n + col] = make_float2(sec.x * bp.x - sec.y * bp.y + c * bq.x, sec.x * bp.y + sec.y * bp.x + c * bq.y);
                }
                a[p * n + q] = make_float2(0.f, 0.f);
                a[q * n + p] = make_float2(0.f, 0.f);
                a[p * n + p] = make_float2(app - t * mag, 0.f);
                a[q * n + q] = make_float2(aqq + t * mag, 0.f);
            }
        }
    }
    // V1: the FP32 columns, orthonormal in FP64 (modified Gram-Schmidt)
    double2 V1[NMAX * NMAX];
    for (int i = 0; i < n * n; ++i) V1[i] = make_double2(v[i].x, v[i].y);
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < j; ++i) {
            double2 r = make_double2(0, 0);
            for (int k = 0; k < n; ++k) r = cfmac(V1[k * n + i], V1[k * n + j], r);   // <v_i, v_j>
            for (int k = 0; k < n; ++k) {
                const double2 t = cmul(r, V1[k * n + i]);
                V1[k * n + j] = make_double2(V1[k * n + j].x - t.x, V1[k * n + j].y - t.y);
            }
        }
        double nrm = 0;
        for (int k = 0; k < n; ++k) nrm += V1[k * n + j].x * V1[k * n + j].x + V1[k * n + j].y * V1[k * n + j].y;
        const double inv = 1.0 / sqrt(nrm);
        for (int k = 0; k < n; ++k) V1[k * n + j] = make_double2(V1[k * n + j].x * inv, V1[k * n + j].y * inv);
    }
    // B = V1^dag A V1 (FP64), into A; V receives T = A V1 first
    for (int r = 0; r < n; ++r)
        for (int j = 0; j < n; ++j) {
            double2 t = make_double2(0, 0);
            for (int k = 0; k < n; ++k) t = cfma(A[r * n + k], V1[k * n + j], t);
            V[r * n + j] = t;
        }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double2 t = make_double2(0, 0);
            for (int k = 0; k < n; ++k) t = cfmac(V1[k * n + i], V[k * n + j], t);
            A[i * n + j] = t;
        }
    // Hermitian to rounding: keep the upper triangle's values on both sides
    for (int i = 0; i < n; ++i) {
        A[i * n + i].y = 0;
        for (int j = i + 1; j < n; ++j) A[j * n + i] = make_double2(A[i * n + j].x, -A[i * n + j].y);
    }
    double2 Q[NMAX * NMAX];
    const int ok = jacobi_hermitian<NMAX>(A, Q, n, w);
    for (int r = 0; r < n; ++r)
        for (int j = 0; j < n; ++j) {
            double2 t = make_double2(0, 0);
            for (int k = 0; k < n; ++k) t = cfma(V1[r * n + k], Q[k * n + j], t);
            V[r * n + j] = t;
        }
    return ok;
}

// Warp-parallel variant for n <= 32 (one warp per matrix, matrices in shared memory with
// row stride ld = n + 1).  The same rotation and stopping rule as jacobi_hermitian, applied in
// the parallel (round-robin) ordering: in each of the n' - 1 rounds of a sweep (n' = n rounded
// up to even), the n'/2 disjoint index pairs are rotated at once.  Disjoint rotations commute,
// and each pair's 2x2 block depends on its own rotation only, so every round zeroes its
// pairs' off-diagonal elements exactly as the sequential sweep does.  Lane r updates row r of
// A and V for the column rotations; lane c updates column c of A for the row rotations.
// Returns 1 on convergence; w receives the eigenvalues in ascending order (lane 0 sorts) and
// V's columns are permuted alike.  All lanes of the warp must call it.
struct JRot {
    int p, q;
    double c, s, ex, ey, app, aqq, tm;
};

__device__ inline int jacobi_hermitian_warp(double2 *A, double2 *V, int n, int ld, double *w,
                                            JRot *rot, int *perm) {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < n; ++j)
        if (lane < n) V[lane * ld + j] = make_double2(lane == j ? 1.0 : 0.0, 0.0);
    __syncwarp();
    const int np = (n + 1) & ~1;          // players of the round robin (one dummy if n is odd)
    int converged = 0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0, tot = 0;
        if (lane < n)
            for (int j = 0; j < n; ++j) {
                const double2 a = A[lane * ld + j];
                const double m2 = a.x * a.x + a.y * a.y;
                tot += m2;
                if (j != lane) off += m2;
            }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if (off <= 1e-30 * tot || off == 0.0) {
            converged = 1;
            break;
        }
        for (int r = 0; r < np - 1; ++r) {
            // pair lane: (np-1, r) for lane 0, ((r+k) mod (np-1), (r-k) mod (np-1)) for lane k
            if (lane < np / 2) {
                int p, q;
                if (lane == 0) {
                    p = np - 1;
                    q = r;
                } else {
                    p = (r + lane) % (np - 1);
                    q = (r - lane + (np - 1)) % (np - 1);
                }
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                JRot R;
                R.p = p;
                R.q = q;
                R.c = 1.0;
                R.s = 0.0;
                R.ex = 1.0;
                R.ey = 0.0;
                R.tm = 0.0;
                R.app = R.aqq = 0.0;
                if (q < n) {                        // a pair with the dummy does nothing
                    const double2 apq = A[p * ld + q];
                    const double mag = sqrt(apq.x * apq.x + apq.y * apq.y);
                    R.app = A[p * ld + p].x;
                    R.aqq = A[q * ld + q].x;
                    if (mag != 0.0) {
                        const double zeta = (R.aqq - R.app) / (2.0 * mag);
                        double t;
                        if (fabs(zeta) > 1e150) t = 0.5 / zeta;
                        else t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                        R.c = 1.0 / sqrt(1.0 + t * t);
                        R.s = t * R.c;
                        R.ex = apq.x / mag;
                        R.ey = apq.y / mag;
                        R.tm = t * mag;
                    } else {
                        R.q = n;                    // nothing to rotate
                    }
                } else {
                    R.q = n;
                }
                rot[lane] = R;
            }
            __syncwarp();
            // columns: A <- A U, V <- V U (lane = row)
            if (lane < n)
                for (int k = 0; k < np / 2; ++k) {
                    const JRot R = rot[k];
                    if (R.q >= n) continue;
                    const double sx = R.s * R.ex, sy = R.s * R.ey;   // s e^{i phi}
                    const double2 ap = A[lane * ld + R.p], aq = A[lane * ld + R.q];
                    A[lane * ld + R.p] = make_double2(R.c * ap.x - (sx * aq.x + sy * aq.y),
                                                      R.c * ap.y - (sx * aq.y - sy * aq.x));
                    A[lane * ld + R.q] = make_double2(sx * ap.x - sy * ap.y + R.c * aq.x,
                                                      sx * ap.y + sy * ap.x + R.c * aq.y);
                    const double2 vp = V[lane * ld + R.p], vq = V[lane * ld + R.q];
                    V[lane * ld + R.p] = make_double2(R.c * vp.x - (sx * vq.x + sy * vq.y),
                                                      R.c * vp.y - (sx * vq.y - sy * vq.x));
                    V[lane * ld + R.q] = make_double2(sx * vp.x - sy * vp.y + R.c * vq.x,
                                                      sx * vp.y + sy * vp.x + R.c * vq.y);
                }
            __syncwarp();
            // rows: A <- U^dag A (lane = column)
            if (lane < n)
                for (int k = 0; k < np / 2; ++k) {
                    const JRot R = rot[k];
                    if (R.q >= n) continue;
                    const double sx = R.s * R.ex, sy = R.s * R.ey;
                    const double2 bp = A[R.p * ld + lane], bq = A[R.q * ld + lane];
                    A[R.p * ld + lane] = make_double2(R.c * bp.x - (sx * bq.x - sy * bq.y),
                                                      R.c * bp.y - (sx * bq.y + sy * bq.x));
                    A[R.q * ld + lane] = make_double2(sx * bp.x + sy * bp.y + R.c * bq.x,
                                                      sx * bp.y - sy * bp.x + R.c * bq.y);
                }
            __syncwarp();
            if (lane < np / 2) {
                const JRot R = rot[lane];
                if (R.q < n) {
                    A[R.p * ld + R.q] = make_double2(0, 0);
                    A[R.q * ld + R.p] = make_double2(0, 0);
                    A[R.p * ld + R.p] = make_double2(R.app - R.tm, 0);
                    A[R.q * ld + R.q] = make_double2(R.aqq + R.tm, 0);
                }
            }
            __syncwarp();
        }
    }
    if (lane == 0) {
        for (int i = 0; i < n; ++i) {
            w[i] = A[i * ld + i].x;
            perm[i] = i;
        }
        for (int i = 0; i < n - 1; ++i) {      // selection sort, ascending
            int k = i;
            for (int j = i + 1; j < n; ++j)
                if (w[j] < w[k]) k = j;
            if (k != i) {
                const double tw = w[i];
                w[i] = w[k];
                w[k] = tw;
                const int tp = perm[i];
                perm[i] = perm[k];
                perm[k] = tp;
            }
        }
    }
    __syncwarp();
    // permute the columns of V (lane = row), through A's row as scratch
    if (lane < n) {
        for (int j = 0; j < n; ++j) A[lane * ld + j] = V[lane * ld + perm[j]];
        for (int j = 0; j < n; ++j) V[lane * ld + j] = A[lane * ld + j];
    }
    __syncwarp();
    return converged;
}
