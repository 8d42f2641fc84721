"""Seeded synthetic inputs for the farPCA tests and benchmark.

Holds none of the method's arithmetic: it only builds the input matrices A that
both the CUDA path and the CPU oracle are run on.  Recipe (arxiv 2506.03859,
Sec. 5, "Matrix 1" / "Matrix 2"): A = U diag(sigma) V^T with U, V Haar
distributed (QR of a seeded standard Gaussian matrix, columns multiplied by the
sign of diag(R)), plus an optional noise term noise * N(0, 1) entrywise.

Spectra (name -> sigma_i, i = 1, 2, ...):
  matrix1   1 / i^2          (Sec. 5, slow decay)
  matrix2   exp(-i / 20)     (Sec. 5, fast decay)
  poly1.5   i^-1.5
  poly1     i^-1
  poly2     i^-2
  exp100    10^(-i / 100)

To keep generation fast, singular values below 1e-18 * sigma_1 are left out
(they change no FP64 entry of A by more than a rounding error of its largest
terms); ``rank`` overrides the number of terms kept.
Arrays are float64 in column-major (Fortran) order, the layout the library
reads.
"""
import numpy as np

SPECTRA = {
    "matrix1": lambda i: 1.0 / i ** 2,
    "matrix2": lambda i: np.exp(-i / 20.0),
    "poly1.5": lambda i: i ** -1.5,
    "poly1": lambda i: 1.0 / i,
    "poly2": lambda i: i ** -2.0,
    "exp100": lambda i: 10.0 ** (-i / 100.0),
}


def singular_values(name, count):
    i = np.arange(1, count + 1, dtype=np.float64)
    return SPECTRA[name](i)


def haar_columns(rows, cols, rng):
    """rows x cols matrix with orthonormal columns, Haar distributed."""
    g = rng.standard_normal((rows, cols))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]


def low_rank_matrix(m, n, spectrum, seed, noise=0.0, rank=None):
    """A = U diag(sigma) V^T (+ noise N(0,1)), float64, column-major."""
    kmax = min(m, n)
    sig = singular_values(spectrum, kmax)
    if rank is None:
        rank = int(np.count_nonzero(sig >= 1e-18 * sig[0]))
    rank = max(1, min(rank, kmax))
    sig = sig[:rank]
    rng = np.random.default_rng(seed)
    U = haar_columns(m, rank, rng)
    V = haar_columns(n, rank, rng)
    A = np.asfortranarray((U * sig[None, :]) @ V.T)
    if noise:
        A += noise * rng.standard_normal((m, n))
    return A


def exact_rank_matrix(m, n, r, seed, spectrum="poly1"):
    """A of exact rank r with distinct singular values (spectrum's first r)."""
    return low_rank_matrix(m, n, spectrum, seed, rank=r)


# Named workloads: the benchmark and parity-test matrices and the paper's Table 1 inputs.
WORKLOADS = {
    # 2000 x 1000, sigma_i = i^-1.5, b = 20, P = 1, eps = 1e-2, zeta = 8
    "dense2000x1000_poly1.5": dict(m=2000, n=1000, spectrum="poly1.5", noise=0.0, seed=1001),
    # 20000 x 10000, sigma_i = 10^(-i/100) + 1e-6 N(0,1) noise, b = 50
    "dense20000x10000_exp100": dict(m=20000, n=10000, spectrum="exp100", noise=1e-6, seed=1002),
    # the same family at a quarter of the size (profiling: A 400 MB, above L2)
    "dense10000x5000_exp100": dict(m=10000, n=5000, spectrum="exp100", noise=1e-6, seed=1003),
    # Table 1, n = 5000
    "matrix1_5000": dict(m=5000, n=5000, spectrum="matrix1", noise=0.0, seed=2001),
    "matrix2_5000": dict(m=5000, n=5000, spectrum="matrix2", noise=0.0, seed=2002),
}


def workload_matrix(name, **override):
    cfg = dict(WORKLOADS[name])
    cfg.update(override)
    return low_rank_matrix(cfg["m"], cfg["n"], cfg["spectrum"], cfg["seed"], cfg.get("noise", 0.0),
                       cfg.get("rank"))


def device_low_rank(m, n, rank, seed, dtype=None, spectrum="exp100", device="cuda", build_dtype=None):
    """A = U diag(sigma) V^T on a CUDA device (torch), column-major, exact rank
    `rank` (U, V with orthonormal columns from QR of seeded Gaussians), built in
    `build_dtype` (default float64) and stored as `dtype` (default float32).  For
    large request pools (the serving workload) and the 60000 x 20000 precision
    workload, where host generation would dominate; building in float32 keeps
    the singular values to ~1e-6 relative, which is all these workloads need."""
    import torch
    dtype = dtype or torch.float32
    build_dtype = build_dtype or torch.float64
    g = torch.Generator(device=device).manual_seed(int(seed))
    U = torch.linalg.qr(torch.randn((m, rank), generator=g, dtype=build_dtype, device=device))[0]
    V = torch.linalg.qr(torch.randn((n, rank), generator=g, dtype=build_dtype, device=device))[0]
    sig = torch.from_numpy(singular_values(spectrum, rank)).to(device=device, dtype=build_dtype)
    A = torch.empty_strided((m, n), (1, m), dtype=dtype, device=device)
    A.copy_((U * sig[None, :]) @ V.T)
    return A


def batch_shapes(count, seed):
    """Shapes of the batched workload: rows uniform in [64, 2048], columns uniform
    in [32, 1024] (independently, so m < n occurs)."""
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(64, 2049)), int(rng.integers(32, 1025))) for _ in range(count)]


def batch_matrix(m, n, seed, rank=64, noise=1e-3, device="cuda"):
    """One problem of the batched workload on the device, float32, column-major:
    U diag(sigma) V^T with sigma_i = i^-2 (i <= min(rank, m, n)), plus Gaussian
    noise of Frobenius norm noise * ||sigma||_2."""
    import torch
    r = min(rank, m, n)
    rng = np.random.default_rng(int(seed))
    U = torch.from_numpy(haar_columns(m, r, rng)).to(device)
    V = torch.from_numpy(haar_columns(n, r, rng)).to(device)
    sig_np = singular_values("poly2", r)
    sig = torch.from_numpy(sig_np).to(device)
    g = torch.Generator(device=device).manual_seed(int(seed))
    A64 = (U * sig[None, :]) @ V.T
    A64 += torch.randn((m, n), generator=g, dtype=torch.float64, device=device) * (
        noise * float(np.linalg.norm(sig_np)) / (m * n) ** 0.5)
    A = torch.empty_strided((m, n), (1, m), dtype=torch.float32, device=device)
    A.copy_(A64)
    return A


def stability_matrix(n, d, seed, device="cuda"):
    """Sec. 5.5's test matrix on the device (float64, column-major): Matrix 1's
    form A = U_A diag(1/i^2) V_A^T with U_A Haar (n x n) and V_A block diagonal,
    d blocks of (n/d) x (n/d), each the orthonormalised factor of a seeded
    Gaussian block (d = n: V_A diagonal with entries +-1; d = 1: V_A dense)."""
    import torch
    assert n % d == 0
    g = torch.Generator(device=device).manual_seed(int(seed))

    def haar(k):
        q, r = torch.linalg.qr(torch.randn((k, k), generator=g, dtype=torch.float64, device=device))
        s = torch.sign(torch.diagonal(r))
        s[s == 0] = 1.0
        return q * s[None, :]

    U = haar(n)
    h = n // d
    if h == 1:
        V = torch.diag(torch.sign(torch.randn(n, generator=g, dtype=torch.float64, device=device)))
    else:
        V = torch.zeros((n, n), dtype=torch.float64, device=device)
        for i in range(d):
            V[i * h:(i + 1) * h, i * h:(i + 1) * h] = haar(h)
    sig = torch.from_numpy(singular_values("matrix1", n)).to(device)
    A = torch.empty_strided((n, n), (1, n), dtype=torch.float64, device=device)
    A.copy_((U * sig[None, :]) @ V.T)
    return A
