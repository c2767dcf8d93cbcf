"""Writes tests/golden/highdim4096_states.npz: FP64 oracle states of Alg. 2 on a
4096 x 4096 sample of the high-dimensional workload, at the iteration counts where
the headline solve is decided.

Calls only ``oracle/`` (the LAMP iteration, Alg. 2 Step 1, and its termination rule
on the infeasibility of X^t, App. E.2) and ``workloads/`` (the seeded points).
No value in the file comes from the CUDA path.

Sample: the first 4096 source and the first 4096 target points of the workload
(n = m = 2^15, d = 64, x ~ N(0, I), y ~ N(0.5 1, I), seed 33), uniform marginals
of size 4096, eta = 0, tau1 = tau2 = 1/(2K), alpha = 0.01, beta = 1.1.

Two problems are run:
  * ``bf16``  the points rounded to bfloat16 (what the tensor-core path multiplies;
              parity tests compare that path with the oracle on this problem);
  * ``fp32``  the float32 points as given (the unrounded problem, against which
              the error of both GPU precisions is reported).
For each, the state (nu^t, theta^t, kappa_t) is stored at t = 500, at t = 1170 (the
headline solve's iteration count at n = 2^15) and at the first t >= 1 whose X^t has
infeasibility <= 1e-6 (t_stop), with <C, X^t> and the infeasibility at t_stop.

Usage:  python tests/golden/make_highdim_states.py [bf16|fp32|merge]
  (bf16 / fp32 write a partial file each; merge combines them; the two runs take
  about 20 minutes each on one core)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "highdim4096_states.npz")
N = 4096
SEED = 33
T_SAVE = (500, 1170)
TOL = 1e-6
MAX_ITER = 4000


def sample_points(variant: str):
    """The 4096 x 4096 sample (float32), rounded to bf16 for variant 'bf16'."""
    w = W.highdim(seed=SEED)
    x = np.ascontiguousarray(w.x[:N])
    y = np.ascontiguousarray(w.y[:N])
    if variant == "bf16":
        x, y = W.bf16_round(x), W.bf16_round(y)
    return x, y


def run(variant: str) -> dict:
    x, y = sample_points(variant)
    C = O.sqeuclid_cost(x, y)
    r = W.uniform_marginal(N)
    c = W.uniform_marginal(N)
    P = O.LampParams()
    K, tau1, tau2 = O.resolve_params(C, P)
    calpha = O.calpha_of(c, P.alpha)
    st = O.lamp_initial_state(N)
    out = {f"{variant}_K": np.float64(K)}
    t0 = time.time()
    while True:
        nxt, info = O.lamp_step(C, r, c, K, tau1, tau2, 0.0, calpha, P.beta, st)
        if st.t in T_SAVE:
            out[f"{variant}_nu_{st.t}"] = st.nu.copy()
            out[f"{variant}_theta_{st.t}"] = st.theta.copy()
            out[f"{variant}_kappa_{st.t}"] = np.float64(st.kappa)
        done = st.t >= 1 and info.res <= TOL
        first = f"{variant}_t_stop" not in out
        if first and (done or st.t >= MAX_ITER):
            out[f"{variant}_nu_stop"] = st.nu.copy()
            out[f"{variant}_theta_stop"] = st.theta.copy()
            out[f"{variant}_kappa_stop"] = np.float64(st.kappa)
            out[f"{variant}_t_stop"] = np.int64(st.t)
            out[f"{variant}_cost_stop"] = np.float64(info.cost_A)
            out[f"{variant}_res_stop"] = np.float64(info.res)
            out[f"{variant}_converged"] = np.bool_(done)
        if f"{variant}_t_stop" in out and st.t >= max(T_SAVE):
            break
        if st.t % 100 == 0:
            print(f"{variant} t={st.t} res={info.res:.3e} ({time.time() - t0:.0f} s)", flush=True)
        st = nxt
    return out


def main():
    what = sys.argv[1] if len(sys.argv) > 1 else "merge"
    if what in ("bf16", "fp32"):
        res = run(what)
        np.savez(os.path.join(HERE, f"_part_{what}.npz"), **res)
        return
    merged = {"n": np.int64(N), "seed": np.int64(SEED), "tol": np.float64(TOL)}
    for v in ("bf16", "fp32"):
        part = os.path.join(HERE, f"_part_{v}.npz")
        with np.load(part) as z:
            merged.update({k: z[k] for k in z.files})
    np.savez_compressed(OUT, **merged)
    for v in ("bf16", "fp32"):
        os.remove(os.path.join(HERE, f"_part_{v}.npz"))
    print("wrote", OUT, os.path.getsize(OUT), "bytes")


if __name__ == "__main__":
    main()
