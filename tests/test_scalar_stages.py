"""The FP64 scalar recurrence of the inner BiCGStab (Alg. 4) as the reducing
kernels run it (csrc/common.cuh: run_stage, the alpha, omega and end-of-
iteration stages, and the norm and rescale-pass stages of Alg. 5), compiled
for the host and compared with the recurrence
written out from its definitions:

  alpha = rho / (r*, v);
  omega = (t, s) / (t, t), and when 0 < |omega^| < omega0 with
  |omega^| = |(t, s)| / (|t| |s|), omega := omega * omega0 / |omega^|;
  with the rescaling of r fused: |s - omega t|^2 from the three sums, floored at
  1e-12 (s, s), and the factor sigma / sqrt of it; x-update coefficients
  (lambda'/gamma') omega and (lambda'/gamma') alpha;
  after the x/r update without fused rescaling: g = |r|, lambda =
  sigma_lambda / |x| (Alg. 5), then the rescale pass's factor sigma / g or the
  end of the iteration with gamma = 1; after the rescale pass: gamma from its
  sums and the earlier g;
  end of iteration: g = |r|, gamma = |r_stored| / g (recalculated) or the
  factor applied, rho' = gamma rho, gamma' *= gamma, lambda' *= lambda
  (Alg. 5), alpha' = alpha,
  omega' = omega, rho = (r*, r_stored), beta = rho alpha' / (rho' omega'),
  p-update coefficients gamma beta and gamma beta omega', |r| / gamma' as the
  residual, and the stopping tests (non-finite, converged, matvec cap,
  breakdown), in that order.

The kernels evaluate some of these with fewer divisions (gamma beta as
rho alpha / (rho_old omega), a reciprocal shared by two products, the omega0
test on squares, sigma times a reciprocal square root). Quantities without
cancellation agree to 2 units in the last place; the cancellation in
|s - omega t|^2 and in the components of gamma beta omega' amplifies the
different roundings to at most ~4e-14 relative over 4000 random cases. The
bound is 1e-12: twelve orders of magnitude below what a wrong term would give."""

import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2602_14450_gb300 import build as B

SRC = r'''
#include "common.cuh"
#include <cstdio>
void wd::tl::register_unit(int (*)(void*, void*)) {}
int main() {
    int stage;
    while (std::scanf("%d", &stage) == 1) {
        double s[4], d[16];
        int iv[8];
        for (double& v : s) std::scanf("%la", &v);
        for (double& v : d) std::scanf("%la", &v);
        for (int& v : iv) std::scanf("%d", &v);
        wd::SolverState st = {};
        st.rho[0] = d[0]; st.rho[1] = d[1]; st.alpha[0] = d[2]; st.alpha[1] = d[3];
        st.omega[0] = d[4]; st.omega[1] = d[5]; st.gamma_p = d[6]; st.lambda_p = d[7]; st.lam = d[8];
        st.sigma = d[9]; st.omega0 = d[10]; st.eps = d[11]; st.bnorm = d[12]; st.gam_tmp = d[13];
        st.g = d[14]; st.sigma_lambda = d[15];
        st.recalc = iv[0]; st.rescale_x = iv[1]; st.fused_scale = iv[2]; st.iter = iv[3]; st.matvecs = iv[4];
        st.max_matvecs = iv[5]; st.status = iv[6]; st.scale_pass = iv[7];
        wd::run_stage(stage, s, &st);
        const double out[] = {st.alpha[0], st.alpha[1], st.omega[0], st.omega[1], st.gam_tmp, st.cXr[0],
                              st.cXr[1], st.cXp[0], st.cXp[1], st.rho_p[0], st.rho_p[1], st.gamma_p,
                              st.alpha_p[0], st.alpha_p[1], st.omega_p[0], st.omega_p[1], st.lambda_p,
                              st.rho[0], st.rho[1], st.cP[0], st.cP[1], st.cV[0], st.cV[1], st.res, st.g,
                              st.lam};
        for (double v : out) std::printf("%a ", v);
        std::printf("%d %d %d %d\n", st.iter, st.matvecs, st.done, st.status);
    }
    return 0;
}
'''
NAMES = ["alpha0", "alpha1", "omega0", "omega1", "gam_tmp", "cXr0", "cXr1", "cXp0", "cXp1", "rho_p0", "rho_p1",
         "gamma_p", "alpha_p0", "alpha_p1", "omega_p0", "omega_p1", "lambda_p", "rho0", "rho1", "cP0", "cP1", "cV0",
         "cV1", "res", "g", "lam"]
ST_ALPHA, ST_OMEGA, ST_RNORM, ST_END, ST_RFUSED = 2, 3, 4, 5, 9
S_OK, S_NOT_CONVERGED, S_BREAKDOWN, S_NONFINITE = 0, 4, 5, 6


@pytest.fixture(scope="module")
def stage_exe():
    d = tempfile.mkdtemp()
    cu, exe = os.path.join(d, "st.cu"), os.path.join(d, "st")
    with open(cu, "w") as f:
        f.write(SRC)
    r = subprocess.run([B.nvcc(), *B.ARCH, *B.FLAGS, "-DWD_TIMELINE", "-I", B.CSRC, cu, "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr)
    return exe


def state(rng, **kw):
    c = lambda: complex(*rng.standard_normal(2))
    st = {"rho": c(), "alpha": c(), "omega": c(), "gamma_p": float(rng.uniform(0.2, 5)),
          "lambda_p": float(rng.uniform(0.5, 2)), "lam": 1.0, "sigma": 64.0, "omega0": 0.7, "eps": 1e-2,
          "bnorm": 128.0, "gam_tmp": float(rng.uniform(0.5, 2)), "recalc": 1, "rescale_x": 0, "fused_scale": 1,
          "iter": int(rng.integers(0, 100)), "matvecs": int(rng.integers(0, 200)), "max_matvecs": 5000,
          "status": S_OK, "g": float(rng.uniform(0.5, 50)), "sigma_lambda": 256.0, "scale_pass": 0}
    st.update(kw)
    return st


def run(exe, cases):
    lines = []
    for stage, s, st in cases:
        d = [st["rho"].real, st["rho"].imag, st["alpha"].real, st["alpha"].imag, st["omega"].real, st["omega"].imag,
             st["gamma_p"], st["lambda_p"], st["lam"], st["sigma"], st["omega0"], st["eps"], st["bnorm"],
             st["gam_tmp"], st["g"], st["sigma_lambda"]]
        iv = [st["recalc"], st["rescale_x"], st["fused_scale"], st["iter"], st["matvecs"], st["max_matvecs"],
              st["status"], st["scale_pass"]]
        lines.append(" ".join([str(stage)] + [float(v).hex() for v in list(s) + d] + [str(v) for v in iv]))
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    res = []
    for line in out.stdout.strip().splitlines():
        w = line.split()
        vals = {n: float.fromhex(v) if not v.endswith("nan") else math.nan for n, v in zip(NAMES, w[:len(NAMES)])}
        vals.update(zip(["iter", "matvecs", "done", "status"], map(int, w[len(NAMES):])))
        res.append(vals)
    return res


def close(a, b, scale=1.0):
    return abs(a - b) <= 1e-12 * max(abs(a), abs(b), scale)


def ref_alpha(s, st):
    v = complex(s[0], s[1])
    if not (math.isfinite(v.real) and math.isfinite(v.imag)):
        return {"done": 1, "status": S_NONFINITE}
    if v == 0:
        return {"done": 1, "status": S_BREAKDOWN}
    a = st["rho"] / v
    return {"alpha0": a.real, "alpha1": a.imag, "done": 0}


def ref_omega(s, st):
    ts, tt, ss = complex(s[0], s[1]), s[2], s[3]
    if not all(math.isfinite(x) for x in (ts.real, ts.imag, tt, ss)):
        return {"done": 1, "status": S_NONFINITE}
    if tt == 0:
        return {"done": 1, "status": S_BREAKDOWN}
    om = ts / tt
    ohat = abs(ts) / math.sqrt(tt * ss) if tt * ss > 0 else math.inf
    if 0 < ohat < st["omega0"]:
        om *= st["omega0"] / ohat
    out = {"omega0": om.real, "omega1": om.imag, "done": 0}
    if st["fused_scale"]:
        r2 = ss - 2 * (om.conjugate() * ts).real + abs(om) ** 2 * tt
        out["gam_tmp"] = st["sigma"] / math.sqrt(max(r2, 1e-12 * ss))
    c = st["lambda_p"] / st["gamma_p"]
    out.update({"cXr0": (c * om).real, "cXr1": (c * om).imag, "cXp0": (c * st["alpha"]).real,
                "cXp1": (c * st["alpha"]).imag})
    return out


def ref_end(s, st):
    """The fused form: sums |r|^2, |r_stored|^2, (r*, r_stored)."""
    r2, rn2, rs = s[0], s[1], complex(s[2], s[3])
    g = math.sqrt(r2)
    gamma = (math.sqrt(rn2) / g if st["recalc"] else st["gam_tmp"]) if r2 != 0 else 1.0
    out = ref_end_iteration(st, gamma, rn2, rs, st["lam"])
    out["g"] = g
    return out


def ref_end_iteration(st, gamma, rn2, rs, lam):
    rho_p = gamma * st["rho"]
    gp = st["gamma_p"] * gamma
    beta = rs * st["alpha"] / (rho_p * st["omega"])
    cp = gamma * beta
    cv = cp * st["omega"]
    res = math.sqrt(rn2) / gp
    mv = st["matvecs"] + 2
    out = {"rho_p0": rho_p.real, "rho_p1": rho_p.imag, "gamma_p": gp, "alpha_p0": st["alpha"].real,
           "lambda_p": st["lambda_p"] * lam if st["rescale_x"] else st["lambda_p"],
           "alpha_p1": st["alpha"].imag, "omega_p0": st["omega"].real, "omega_p1": st["omega"].imag,
           "rho0": rs.real, "rho1": rs.imag, "cP0": cp.real, "cP1": cp.imag, "cV0": cv.real, "cV1": cv.imag,
           "res": res, "iter": st["iter"] + 1, "matvecs": mv}
    if res <= st["eps"] * st["bnorm"]:
        out.update(done=1, status=S_OK)
    elif mv >= st["max_matvecs"]:
        out.update(done=1, status=S_NOT_CONVERGED)
    else:
        out.update(done=0)
    return out


def check(got, want, case):
    for k, v in want.items():
        if k in ("done", "status", "iter", "matvecs"):
            assert got[k] == v, (case, k, got[k], v)
        else:
            assert close(got[k], v), (case, k, got[k], v)


def test_alpha_stage(stage_exe):
    rng = np.random.default_rng(31)
    cases = [(ST_ALPHA, [*rng.standard_normal(2) * 10.0 ** rng.integers(-8, 8), 0, 0], state(rng)) for _ in range(200)]
    cases += [(ST_ALPHA, [0.0, 0.0, 0, 0], state(rng)), (ST_ALPHA, [math.nan, 1.0, 0, 0], state(rng)),
              (ST_ALPHA, [math.inf, 0.0, 0, 0], state(rng))]
    for (stage, s, st), got in zip(cases, run(stage_exe, cases)):
        check(got, ref_alpha(s, st), (s, st))


def test_omega_stage(stage_exe):
    rng = np.random.default_rng(32)
    cases = []
    for i in range(400):
        tt, ss = float(rng.uniform(0.1, 1e4)), float(rng.uniform(0.1, 1e4))
        c = float(rng.uniform(0.01, 1.0))           # |(t, s)| / (|t| |s|): below and above omega0 = 0.7
        phi = float(rng.uniform(0, 2 * math.pi))
        ts = c * math.sqrt(tt * ss) * complex(math.cos(phi), math.sin(phi))
        cases.append((ST_OMEGA, [ts.real, ts.imag, tt, ss], state(rng, fused_scale=int(i % 2), omega0=[0.7, 0.0][i % 3 == 0])))
    cases += [(ST_OMEGA, [1.0, 0.0, 0.0, 1.0], state(rng)), (ST_OMEGA, [math.nan, 0.0, 1.0, 1.0], state(rng)),
              (ST_OMEGA, [0.0, 0.0, 2.0, 3.0], state(rng))]
    for (stage, s, st), got in zip(cases, run(stage_exe, cases)):
        check(got, ref_omega(s, st), (s, st))


def test_end_of_iteration_stage(stage_exe):
    rng = np.random.default_rng(33)
    cases = []
    for i in range(400):
        r2 = float(rng.uniform(1e-6, 1e6))
        rn2 = float(rng.uniform(1e-6, 1e6))
        rs = complex(*rng.standard_normal(2)) * 10.0 ** float(rng.integers(-3, 3))
        kw = {"recalc": int(i % 2)}
        if i % 7 == 0:
            kw.update(eps=1e9)                      # converged
        if i % 11 == 0:
            kw.update(matvecs=4998)                 # reaches the cap
        cases.append((ST_RFUSED, [r2, rn2, rs.real, rs.imag], state(rng, **kw)))
    cases.append((ST_RFUSED, [0.0, 0.0, 0.0, 0.0], state(rng)))   # r = 0 exactly: gamma = 1, converged
    for (stage, s, st), got in zip(cases, run(stage_exe, cases)):
        check(got, ref_end(s, st), (s, st))


def ref_rnorm(s, st):
    """Norms after the x/r update without fused rescaling: |r|^2, |x|^2, (r*, r); then either the rescale pass's
    factor (Alg. 5 with its separate pass) or the end of the iteration with gamma = 1."""
    r2, x2, rs = s[0], s[1], complex(s[2], s[3])
    g = math.sqrt(r2)
    lam = st["sigma_lambda"] / math.sqrt(x2) if st["rescale_x"] else st["lam"]
    if st["scale_pass"]:
        gt = st["sigma"] / g if st["sigma"] > 0 else 1.0
        out = {"g": g, "gam_tmp": gt, "lam": lam, "done": 0}
        if not math.isfinite(gt) or (st["rescale_x"] and not math.isfinite(lam)):
            out.update(done=1, status=S_NONFINITE)
        return out
    out = ref_end_iteration(st, 1.0, r2, rs, lam)
    out.update(g=g, lam=lam)
    return out


def ref_end_after_scale(s, st):
    """After the rescale pass (Alg. 5): |r_stored|^2, (r*, r_stored); gamma from the g of the norms' stage."""
    rn2, rs = s[0], complex(s[1], s[2])
    gamma = (math.sqrt(rn2) / st["g"] if st["recalc"] else st["gam_tmp"]) if st["sigma"] > 0 else 1.0
    return ref_end_iteration(st, gamma, rn2, rs, st["lam"])


def test_norm_and_rescale_pass_stages(stage_exe):
    rng = np.random.default_rng(34)
    cases = []
    for i in range(400):
        r2, x2 = float(rng.uniform(1e-4, 1e6)), float(rng.uniform(1e-4, 1e6))
        rs = complex(*rng.standard_normal(2))
        kw = {"rescale_x": int(i % 2), "scale_pass": int((i // 2) % 2), "lam": float(rng.uniform(0.5, 2)),
              "sigma": [64.0, 0.0][i % 5 == 0]}
        cases.append((ST_RNORM, [r2, x2, rs.real, rs.imag], state(rng, **kw)))
    for i in range(400):
        rn2 = float(rng.uniform(1e-4, 1e6))
        rs = complex(*rng.standard_normal(2))
        kw = {"rescale_x": int(i % 2), "recalc": int((i // 2) % 2), "lam": float(rng.uniform(0.5, 2)),
              "sigma": [64.0, 0.0][i % 5 == 0]}
        if i % 7 == 0:
            kw.update(eps=1e9)
        cases.append((ST_END, [rn2, rs.real, rs.imag, 0.0], state(rng, **kw)))
    for (stage, s, st), got in zip(cases, run(stage_exe, cases)):
        check(got, ref_rnorm(s, st) if stage == ST_RNORM else ref_end_after_scale(s, st), (stage, s, st))
