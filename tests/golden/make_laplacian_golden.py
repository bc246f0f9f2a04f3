"""Writes laplacian_eigs_n8.txt: the closed-form eigenvalues of the 1D Dirichlet
FD Laplacian printed in Section 3.5 ("eig_lap"), with the sign read for -Delta:
lambda_k = (4/h^2) sin^2(pi k h / 2), h = 1/(n+1), k = 1..n. Evaluates the
printed formula only (no oracle or library code)."""
import math
import os

n = 8
h = 1.0 / (n + 1)
vals = [4.0 / h ** 2 * math.sin(math.pi * k * h / 2.0) ** 2 for k in range(1, n + 1)]
path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "laplacian_eigs_n8.txt")
with open(path, "w") as f:
    f.write("# closed form (Section 3.5, eig_lap): lambda_k = 4/h^2 sin^2(pi k h/2), n=8, h=1/9\n")
    for v in vals:
        f.write(f"{v:.17e}\n")
