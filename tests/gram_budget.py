"""Error budget of the tensor-core Gram matrices (a helper of the GPU parity tests).

The mixed path forms G = X^T Y on the tensor cores from float32 values (each the
float64 value rounded to nearest) written as three integer digits below 2^E,
the power of two above the largest |value| of its column over a chunk of 128
consecutive padded-grid nodes.  The only error is that rounding to a grid of
2^(E - 24): at most 2^(E - 25) per value, unbiased, so with independent errors
a Gram entry is off by a zero-mean sum whose variance is
    sum_k (var(dx_k) y_k^2 + x_k^2 var(dy_k)),  var = 2^(2E - 48) / 12,
and every other step (the exact digit products, the float-float accumulation)
adds nothing at this level; the products of digit levels >= 3, which the kernel
drops, are zero-mean terms of the same order and at most double the variance.
gram_tc_error returns the expected largest deviation over the N x N entries:
the largest standard deviation times sqrt(2 ln N^2) (the extreme value of N^2
zero-mean Gaussian errors) times sqrt(2).  Through the small eigenproblem (C the
G_B-orthonormal eigenvectors, ||C||^2 = 1 / lambda_min(G_B)) an entry of
U^T M U - I = -C^T dG_B C, or a Ritz value's shift c^T (dG_A - theta dG_B) c,
is a weighted sum of these entry errors and inherits that size times ||C||^2.
(A numpy emulation of the digit scheme on a 32^3 oscillator block, N = 20: largest
entry error 1.4e-8 against an expected 1.9e-8 by this formula.)
"""
import numpy as np


def padded_index(n):
    """Padded-grid node index of every interior node, in unknown order (x fastest)."""
    nx, ny, nz = n
    Px, Py = nx + 1, ny + 1
    k, j, i = np.meshgrid(np.arange(1, nz), np.arange(1, ny), np.arange(1, nx), indexing="ij")
    return ((k * Py + j) * Px + i).ravel()


def _grid_step_var(A, chunk):
    """Per value: variance of its rounding to 2^(E - 24), E from its column's chunk maximum."""
    nch = int(chunk.max()) + 1
    cmax = np.zeros((nch, A.shape[1]))
    np.maximum.at(cmax, chunk, np.abs(A))
    E = np.where(cmax > 0, np.floor(np.log2(np.where(cmax > 0, cmax, 1.0))) + 1.0, 0.0)
    step = np.where(cmax > 0, 2.0 ** (E - 24), 0.0)
    return (step ** 2 / 12.0)[chunk]


def gram_tc_error(n, X, Y):
    """Expected largest entry error of the tensor-core X^T Y (float64 inputs)."""
    chunk = padded_index(n) // 128
    vx, vy = _grid_step_var(X, chunk), _grid_step_var(Y, chunk)
    var = vx.T @ (Y ** 2) + (X ** 2).T @ vy
    entries = X.shape[1] * Y.shape[1]
    return float(np.sqrt(2.0 * np.max(var)) * np.sqrt(2.0 * np.log(max(entries, 2))))


def rotation_tc_error(X, C, MU, blk=128):
    """Expected largest entry error of U^T M U added by the tensor-core rotation U = X C.

    The rotation runs in blocks of at most `blk` orbitals along K (the columns of X,
    the rows of C): within a block it rounds every X row to 24 bits below its
    largest |value| over the block and every C column to 24 bits below its largest
    |value| over the block's rows, to nearest; dU = dX C + X dC has per-entry
    variances var_U[g, i] = sum_a (var(dX_ga) C_ai^2 + X_ga^2 var(dC_ai)), and
    (U + dU)^T M (U + dU) - U^T M U ~ dU^T M U + U^T M dU has entry variances
    sum_g (var_U[g, i] MU_gj^2 + var_U[g, j] MU_gi^2).  Returned: the largest
    standard deviation times sqrt(2 ln N^2), as gram_tc_error.
    """
    def step2(A, axis):
        amax = np.max(np.abs(A), axis=axis, keepdims=True)
        E = np.where(amax > 0, np.floor(np.log2(np.where(amax > 0, amax, 1.0))) + 1.0, 0.0)
        return np.where(amax > 0, 2.0 ** (2 * (E - 24)) / 12.0, 0.0)

    varU = np.zeros((X.shape[0], C.shape[1]))
    for k0 in range(0, C.shape[0], blk):
        Xb, Cb = X[:, k0:k0 + blk], C[k0:k0 + blk, :]
        vx = step2(Xb, 1)  # per node row of the block
        vc = step2(Cb, 0)  # per column of the block
        varU += vx * np.sum(Cb ** 2, axis=0)[None, :] + (Xb ** 2) @ np.broadcast_to(vc, Cb.shape)
    var = varU.T @ (MU ** 2) + (MU ** 2).T @ varU
    N = C.shape[1]
    return float(np.sqrt(np.max(var)) * np.sqrt(2.0 * np.log(max(N * N, 2))))
