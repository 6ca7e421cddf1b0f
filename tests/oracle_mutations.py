"""Mutation check of the oracle's pins (test infrastructure, CPU only; not collected by pytest).

Plants one plausible mistake at a time in a scratch copy of oracle/ (a wrong constant, bit, scale,
index order or sign; a dropped term; a transposed operand), runs the CPU pins
(tests/test_oracle_*.py and tests/test_row_shards.py) against it, and lists the mistakes that no
pin catches. Usage: python tests/oracle_mutations.py [index ...]   (exit status 1 if any survive)
"""
import os
import shutil
import subprocess
import sys
import tempfile

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MUTS = [
    ("rng.py", "(c + np.uint64(1)) * _GOLDEN", "c * _GOLDEN", "splitmix counter offset"),
    ("rng.py", "z = z ^ (z >> np.uint64(31))", "z = z ^ (z >> np.uint64(30))", "splitmix final shift"),
    ("rng.py", "b = ((x >> np.uint64(32)) * np.uint64(s)) >> np.uint64(32)\n    sign",
     "b = ((x & np.uint64(0xFFFFFFFF)) * np.uint64(s)) >> np.uint64(32)\n    sign", "bucket from low word"),
    ("rng.py", "    sign = np.where((x & np.uint64(1)) == 0, 1.0, -1.0)\n    return b",
     "    sign = np.where((x & np.uint64(2)) == 0, 1.0, -1.0)\n    return b", "sign from bit 1"),
    ("rng.py", "np.cos(2.0 * np.pi * u2)", "np.sin(2.0 * np.pi * u2)", "Box-Muller sine branch"),
    ("rng.py", ".astype(np.float64) + 1.0) * 2.0 ** -53", ".astype(np.float64) + 0.5) * 2.0 ** -53", "u1 offset"),
    ("rng.py", "bf16_round(gaussian(seed, STREAM_G, counters)) / np.sqrt(m)",
     "bf16_round(gaussian(seed, STREAM_G, counters)) / m", "G scaled by 1/m"),
    ("rng.py", "return gaussian(seed, STREAM_OMEGA, idx) / np.sqrt(k)", "return gaussian(seed, STREAM_OMEGA, idx) / k",
     "Omega scaled by 1/k"),
    ("rng.py", "(bits + np.uint64(0x7FFF) + ((bits >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)",
     "(bits) & np.uint64(0xFFFF0000)", "BF16 truncation"),
    ("rng.py", "idx = j * np.uint64(s) + b", "idx = b * np.uint64(m) + j", "G counter order"),
    ("rng.py", "idx = np.arange(r * k, dtype=np.uint64).reshape(r, k)",
     "idx = np.arange(r * k, dtype=np.uint64).reshape(k, r).T", "Omega counter order"),
    ("rng.py", "return (((x >> np.uint64(32)) * np.uint64(s)) >> np.uint64(32)).astype(np.int64)",
     "return ((x >> np.uint64(32)) % np.uint64(s)).astype(np.int64)", "SRHT rows by modulo"),
    ("estimator.py", "S = sp.csr_matrix((sign, (b, np.arange(r1 - r0)))",
     "S = sp.csr_matrix((np.abs(sign), (b, np.arange(r1 - r0)))", "CountSketch signs dropped"),
    ("estimator.py", "start=row0 + r0", "start=r0", "row0 ignored"),
    ("estimator.py", "Y[:, 1] = a - Y[:, 1]", "Y[:, 1] = Y[:, 1] - a", "FWHT butterfly sign"),
    ("estimator.py", "return X[rng.srht_rows(t, s, seed)] / np.sqrt(t)",
     "return X[rng.srht_rows(t, s, seed)] / np.sqrt(s)", "SRHT scale"),
    ("estimator.py", "Om = np.eye(r) if omega_identity else rng.omega(r, k, seed)",
     "Om = np.eye(r) if omega_identity else rng.omega(r, k, seed + 1)", "Omega seed"),
    ("estimator.py", "out[np.asarray(perm[:r])] = M", "out[np.sort(np.asarray(perm[:r]))] = M", "Mfull rows sorted"),
    ("estimator.py", "theta[r0:r0 + block] = np.sum(Y * Y, axis=1)",
     "theta[r0:r0 + block] = np.sum(Y, axis=1) ** 2", "row norm as squared sum"),
    ("estimator.py", "cols = np.asarray(perm[:r], dtype=np.int64)",
     "cols = np.sort(np.asarray(perm[:r], dtype=np.int64))", "final pass columns sorted"),
    ("linalg.py", "p = ties[np.argmin(perm[ties])]", "p = ties[np.argmax(perm[ties])]", "ties to highest index"),
    ("linalg.py", "if best == 0.0 or best <= tau * r00:", "if best == 0.0 or best <= tau * tau * r00:",
     "rank test tau^2"),
    ("linalg.py", "R[j, j:] = sgn * W[j, j:]", "R[j, j:] = W[j, j:]", "no sign normalisation"),
    ("linalg.py", "R[:j, [j, p]] = R[:j, [p, j]]", "R[:j, [j, p]] = R[:j, [j, p]]", "R rows not swapped"),
    ("linalg.py", "X[p] = (B[p] - R11[p, p + 1:] @ X[p + 1:]) / R11[p, p]",
     "X[p] = (B[p] - R11[p + 1:, p] @ X[p + 1:]) / R11[p, p]", "back-substitution transposed"),
    ("exact.py", "keep = lam > (tau * tau) * lam[0]", "keep = lam > tau * lam[0]", "Gram rank tau not tau^2"),
    ("exact.py", "            Gm += blk.T @ blk\n", "            Gm = blk.T @ blk\n", "Gram blocks not summed"),
    ("exact.py", "X = V / np.sqrt(lam)[None, :]", "X = V / lam[None, :]", "Alg. 7 Sigma^-2"),
    ("rank.py", "return int(np.sum(sigma > zeta * sigma[0]))", "return int(np.sum(sigma > zeta * zeta * sigma[0]))",
     "SVD rank zeta^2"),
    ("rank.py", "rho = np.sqrt(X ** 2 + (gamma[None, :] * inv_omega[:, None]) ** 2)", "rho = np.abs(X)",
     "SRRQR gamma term dropped"),
    ("rank.py", "perm[i], perm[k + j] = perm[k + j], perm[i]", "perm[i], perm[j] = perm[j], perm[i]",
     "SRRQR swap index"),
    ("precond.py", "N = Vt[:k].T / sig[:k][None, :]", "N = Vt[:k].T * sig[:k][None, :]", "N = V Sigma"),
    ("precond.py", "rhobar = -c * alpha", "rhobar = c * alpha", "LSQR rhobar sign"),
    ("precond.py", "w = v - (theta / rho) * w", "w = v + (theta / rho) * w", "LSQR w update sign"),
    ("precond.py", "return (1 + alpha + q) / (1 - alpha - q)", "return (1 + alpha + q) / (1 - alpha + q)",
     "xi denominator"),
    ("backward.py", "return np.tril(X) + np.tril(X, -1).T", "return np.triu(X) + np.triu(X, 1).T", "copyltu upper"),
    ("backward.py", "Z = 2.0 * w[:, None] * Y", "Z = w[:, None] * Y", "adjoint factor 2"),
    ("backward.py", "return 2.0 * (np.eye(n) - H)", "return 2.0 * (np.eye(n) + H)", "exact gradient I + H"),
    ("backward.py", "Rbar = -solve_triangular", "Rbar = solve_triangular", "Rbar sign"),
    ("backward.py", "T_rows = sign[:, None] * Gt[b]", "T_rows = Gt[b]", "S^T signs dropped"),
    ("estimator.py", "At += rng.gaussian_sketch_block(m, s, seed, c0, c1) @ B[c0:c1]",
     "At = rng.gaussian_sketch_block(m, s, seed, c0, c1) @ B[c0:c1]", "Gaussian-stage blocks not summed"),
    ("estimator.py", "B += prod.toarray() if sp.issparse(prod) else prod",
     "B = prod.toarray() if sp.issparse(prod) else prod", "CountSketch blocks not summed"),
    ("rank.py", "sgn = np.where(np.diag(R) < 0, -1.0, 1.0)", "sgn = np.ones(R.shape[0])", "r_factor signs"),
    ("precond.py", "k = rank_svd(sig, zeta)", "k = rank_svd(sig, zeta * zeta)", "Alg. 11 rank zeta^2"),
    ("precond.py", "phibar * alpha * abs(c) <= atol", "phibar * alpha * c <= atol", "LSQR stop without |c|"),
    ("precond.py", "bnorm2 += alpha * alpha + beta * beta", "bnorm2 += alpha * alpha", "LSQR norm estimate"),
    ("exact.py", "B = gram(A_K, block)", "B = gram(A, block)", "Alg. 7 Gram of all columns"),
    ("exact.py", "Q = qr.q_thin(qr.rank)", "Q = qr.q_thin(max(qr.rank - 1, 1))", "thin Q one column short"),
    ("linalg.py", "return Q * self._signs[None, :cols]", "return Q", "thin Q signs"),
    ("rng.py", "    return np.where((x & np.uint64(1)) == 0, 1.0, -1.0)\n\n\ndef srht_rows",
     "    return np.where((x & np.uint64(2)) == 0, 1.0, -1.0)\n\n\ndef srht_rows", "SRHT sign bit"),
    ("rng.py", "return (int(seed) ^ ((stream * _STREAM_MUL) & _MASK64)) & _MASK64",
     "return (int(seed) + ((stream * _STREAM_MUL) & _MASK64)) & _MASK64", "stream key by addition"),
    ("estimator.py", "forced_perm = rank_mod.srrqr(Atilde, forced_rank, srrqr_phi, forced_perm)[0]",
     "forced_perm = rank_mod.srrqr(Atilde, max(forced_rank - 1, 0), srrqr_phi, forced_perm)[0]",
     "Alg. 10 SRRQR at rank - 1"),
    ("estimator.py", "forced_rank = rank_mod.rank_svd(rank_mod.singular_values(Atilde), tau)",
     "forced_rank = rank_mod.rank_svd(rank_mod.singular_values(Atilde.T @ Atilde), tau)",
     "SVD rule on the Gram matrix"),
    ("linalg.py", "trailing = np.sqrt(np.sum(W[j:, j:] ** 2, axis=0))",
     "trailing = np.sqrt(np.sum(W[:, j:] ** 2, axis=0))", "trailing norms include eliminated rows"),
    ("exact.py", "X = V[:, :k] / np.sqrt(lam[:k])[None, :]", "X = V[:, :k] * np.sqrt(lam[:k])[None, :]",
     "Gram route scaled the wrong way"),
    ("estimator.py", "X = fwht(rng.srht_signs(s, seed)[:, None] * B)",
     "X = rng.srht_signs(s, seed)[:, None] * fwht(B)", "SRHT as D H instead of H D"),
    ("backward.py", 'C @ M.T, lower=False, trans="T")', 'C @ M.T, lower=False, trans="N")',
     "adjoint solve not transposed"),
    ("rng.py", "return gaussian(seed, STREAM_OMEGA, idx) / np.sqrt(k)",
     "return gaussian(seed, STREAM_G, idx) / np.sqrt(k)", "Omega from the G stream"),
    ("exact.py", "order = np.argsort(lam)[::-1]", "order = np.argsort(lam)", "Gram eigenvalues ascending"),
    ("backward.py", "    Om = np.eye(r) if omega_identity else rng.omega(r, k, seed)\n    M = solve_triangular(R11, Om, lower=False)\n    Y = AK @ M\n    return",
     "    Om = np.eye(r) if omega_identity else rng.omega(r, k, seed)\n    M = solve_triangular(R11.T, Om, lower=True)\n    Y = AK @ M\n    return",
     "theta_fixed solves with R^T"),
    ("rank.py", "dets.append(float(np.prod(np.abs(np.diag(R)[:k]))))",
     "dets.append(float(np.prod(np.abs(np.diag(R)[:k + 1]))))", "SRRQR det over k + 1"),
    ("rng.py", "np.arange(start, start + n, dtype=np.uint64))", "np.arange(n, dtype=np.uint64))", "hash ignores start"),
    ("linalg.py", "Q[j:, :] -= np.outer(v, beta * (v @ Q[j:, :]))", "Q[j:, :] += np.outer(v, beta * (v @ Q[j:, :]))",
     "thin Q reflector sign"),
]


def main():
    tmp = tempfile.mkdtemp(prefix="mut_")
    for name in ("oracle", "tests", "workloads", "paper_2105_11004_gb300", "include"):
        shutil.copytree(os.path.join(REPO, name), os.path.join(tmp, name),
                        ignore=shutil.ignore_patterns("__pycache__", "_build"))
    shutil.copy(os.path.join(REPO, "__graft_entry__.py"), tmp)
    tests = sorted(f"tests/{f}" for f in os.listdir(os.path.join(REPO, "tests"))
                   if f.startswith("test_oracle") or f == "test_row_shards.py")
    base = {f: open(os.path.join(REPO, "oracle", f)).read() for f in os.listdir(os.path.join(REPO, "oracle"))
            if f.endswith(".py")}
    only = set(sys.argv[1:])
    survivors = []
    for i, (f, old, new, what) in enumerate(MUTS):
        if only and str(i) not in only:
            continue
        src = base[f]
        if src.count(old) < 1:
            print(f"[{i}] {what}: pattern not found")
            survivors.append((i, what, "pattern not found"))
            continue
        for g, s in base.items():
            open(os.path.join(tmp, "oracle", g), "w").write(s)
        open(os.path.join(tmp, "oracle", f), "w").write(src.replace(old, new, 1))
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"] + tests,
                           cwd=tmp, capture_output=True, text=True, timeout=900)
        caught = r.returncode != 0
        last = [l for l in r.stdout.splitlines() if "failed" in l or "passed" in l or "error" in l.lower()][-1:]
        print(f"[{i}] {what}: {'caught' if caught else 'SURVIVED'} {last}", flush=True)
        if not caught:
            survivors.append((i, what, ""))
    shutil.rmtree(tmp, ignore_errors=True)
    print("survivors:", survivors)
    return 1 if survivors else 0


if __name__ == "__main__":
    sys.exit(main())
