"""Target runs of the stability method on the GPU, verified by the oracle.

Not collected by pytest (a GPU run of minutes): run it on a GB300 as
    python tests/target_runs.py --n 100 --alpha 0 --path 300,600,...,1900 \
        --eig-re 1900 --m 60 --nev 10 --out result.json

Steps (Section 3):
1. steady states by Newton continuation in Re from rest (or from a saved
   state) on the n^3 grid (newton_steady, float-float Krylov vectors, the
   Stokes-type right preconditioner of the corrections, ||F||_inf < tol);
   each stage starts from the secant extrapolation of the last two
   converged states, and a failed stage is retried at half the Re step;
2. at each Re of --eig-re the leading eigenvalues by implicitly restarted
   Arnoldi in regular mode (arnoldi_leading) from the seeded Gaussian start
   vector;
3. optional: the critical Re by the secant method on Re(Lambda) from the two
   Re of --secant (fv_critical_re);
4. verification with the FP64 oracle (CPU): the steady residual
   oracle.krylov.steady_residual of the device steady state, and the
   eigen-residual ||A x - lambda x||_W / |lambda| of the leading Ritz pair
   with A the oracle's Krylov vector (exact projection) in its shifted
   form, both computed from the device fields.
Wall times are taken around each library call, synchronised.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=48)
    ap.add_argument("--map", default="cosine")
    ap.add_argument("--alpha", type=float, default=0.0, help="lid angle in degrees")
    ap.add_argument("--path", default="300,600,900,1200,1500,1800,1900")
    ap.add_argument("--eig-re", default="1900")
    ap.add_argument("--secant", default="", help="re0,re1 of a critical-Re secant search")
    ap.add_argument("--secant-rtol", type=float, default=1e-6)
    ap.add_argument("--m", type=int, default=60)
    ap.add_argument("--nev", type=int, default=10)
    ap.add_argument("--prec", default="ff")
    ap.add_argument("--newton-tol", type=float, default=1e-10)
    ap.add_argument("--arnoldi-tol", type=float, default=1e-8)
    ap.add_argument("--max-restarts", type=int, default=20000)
    ap.add_argument("--precond", type=int, default=1)
    ap.add_argument("--linear", default="gmres+bicgstab")
    ap.add_argument("--gmres-m", type=int, default=100)
    ap.add_argument("--gmres-rtol", type=float, default=1e-8)
    ap.add_argument("--gmres-sat", type=float, default=0.5)
    ap.add_argument("--max-newton", type=int, default=30)
    ap.add_argument("--precond-sigma", type=float, default=0.0)
    ap.add_argument("--load-re", type=float, default=0.0, help="Re of the --load state")
    ap.add_argument("--predictor", type=int, default=1, help="secant predictor in Re")
    ap.add_argument("--forcing", type=int, default=0, help="1: Eisenstat-Walker linear tolerances")
    ap.add_argument("--gmres-aug", type=int, default=0, help="augmentation vectors of flexible GMRES")
    ap.add_argument("--tau", type=float, default=0.0, help="shift of the Newton corrections")
    ap.add_argument("--halvings", type=int, default=3, help="Re-step halvings after a failed stage")
    ap.add_argument("--load", default="", help=".npy velocity to start the continuation from")
    ap.add_argument("--save", default="", help="write the last converged velocity here (.npy)")
    ap.add_argument("--save-at", default="", help="Re values whose states also go to --save-pattern")
    ap.add_argument("--save-evec", default="", help="write the leading eigenvector (re, im) here (.npy)")
    ap.add_argument("--save-pattern", default="", help="path with {re}")
    ap.add_argument("--verify", type=int, default=1)
    ap.add_argument("--out", default="target_run.json")
    a = ap.parse_args()

    import torch
    import paper_1704_08521_gb300 as fv
    import synth

    n = a.n
    alpha = np.deg2rad(a.alpha)
    path = [float(x) for x in a.path.split(",") if x]
    eig_re = [float(x) for x in a.eig_re.split(",") if x]
    res = {"n": n, "map": a.map, "alpha_deg": a.alpha, "prec": a.prec, "precond": a.precond,
           "linear": a.linear, "gmres_m": a.gmres_m, "gmres_rtol": a.gmres_rtol, "load": a.load,
           "precond_sigma": a.precond_sigma, "forcing": a.forcing, "predictor": a.predictor,
           "gmres_aug": a.gmres_aug, "tau": a.tau,
           "newton": [], "arnoldi": [], "critical": None, "verify": {}}
    dev = torch.device("cuda")
    g = fv.Grid(n, n, n, a.map, alpha=alpha, re=path[0])
    U = torch.zeros(g.n_vel, dtype=torch.float64, device=dev)
    if a.load:
        U.copy_(torch.from_numpy(np.load(a.load)))
    P = torch.zeros(g.n_cell, dtype=torch.float64, device=dev)
    v0 = torch.tensor(synth.gaussian_velocity((n, n, n), 1), device=dev)
    evec = torch.empty(2 * g.n_vel, dtype=torch.float64, device=dev)
    states = {}

    def sync_time():
        torch.cuda.synchronize()
        return time.perf_counter()

    # continuation: a secant predictor from the last two converged states,
    # and a halved Re step (up to --halvings times) after a failed stage
    conv = []                                   # (re, U) of the last converged states
    if a.load:
        conv.append((a.load_re, U.clone()))
    queue = list(path)
    halvings = 0
    while queue:
        re = queue[0]
        g.set_re(re)
        U_prev = U.clone()
        if len(conv) >= 2 and a.predictor:
            (r0, U0), (r1, U1) = conv[-2], conv[-1]
            U.copy_(U1 + (U1 - U0) * ((re - r1) / (r1 - r0)))
        t0 = sync_time()
        st = fv.newton_steady(g, U, P, tol=a.newton_tol, prec=a.prec, precond=a.precond,
                              precond_sigma=a.precond_sigma, forcing=a.forcing,
                              gmres_aug=a.gmres_aug, tau=a.tau, linear=a.linear, gmres_m=a.gmres_m, gmres_sat=a.gmres_sat,
                              gmres_max_it=20000, gmres_rtol=a.gmres_rtol, max_newton=a.max_newton,
                              raise_on_fail=False)
        t1 = sync_time()
        rec = {"re": re, "s": t1 - t0, "status": st["status"], "steps": st["iterations"],
               "products": st["gmres_total"] + st["bicgstab_total"], "res": st["res_hist"],
               "lin": st["lin_hist"], "predicted": len(conv) >= 2 and a.predictor}
        res["newton"].append(rec)
        print(json.dumps(rec), flush=True)
        if st["status"] != 0:
            U.copy_(U_prev)
            if halvings < a.halvings and conv:
                halvings += 1
                queue.insert(0, 0.5 * (conv[-1][0] + re))
                continue
            break
        queue.pop(0)
        if re in path:
            halvings = 0
        conv = (conv + [(re, U.clone())])[-2:]
        if a.save:
            np.save(a.save, U.cpu().numpy())
        if a.save_pattern and re in [float(x) for x in a.save_at.split(",") if x]:
            np.save(a.save_pattern.replace("{re}", f"{re:g}"), U.cpu().numpy())
        if re in eig_re:
            states[re] = U.clone()
            t0 = sync_time()
            try:
                lam, info = fv.arnoldi_leading(g, U, v0, m=a.m, nev=a.nev, evec=evec, prec=a.prec,
                                               tol=a.arnoldi_tol, max_restarts=a.max_restarts)
                ok = True
            except fv.FvError as e:
                lam, info, ok = [], {"error": str(e)}, False
            t1 = sync_time()
            rec = {"re": re, "s": t1 - t0, "ok": ok,
                   "lambda": [[z.real, z.imag] for z in lam], "info": info}
            res["arnoldi"].append(rec)
            print(json.dumps(rec), flush=True)
            if ok:
                states[("evec", re)] = (evec.clone(), lam[0])
                if a.save_evec:
                    np.save(a.save_evec, evec.cpu().numpy())
    if a.secant and res["newton"] and res["newton"][-1]["status"] == 0:
        r0, r1 = [float(x) for x in a.secant.split(",")]
        t0 = sync_time()
        try:
            rc, om, hist = fv.fv_critical_re(g, U, P, v0, r0, r1, rtol=a.secant_rtol, m=a.m,
                                             nev=a.nev, prec=a.prec, newton_tol=a.newton_tol,
                                             arnoldi_tol=a.arnoldi_tol, precond=a.precond,
                                             precond_sigma=a.precond_sigma, forcing=a.forcing,
                                             max_restarts=a.max_restarts, tau=a.tau,
                                             max_newton=a.max_newton)
            res["critical"] = {"re_cr": rc, "omega_cr": om, "hist": hist}
        except fv.FvError as e:
            res["critical"] = {"error": str(e)}
        res["critical"]["s"] = sync_time() - t0
        print(json.dumps(res["critical"]), flush=True)
    if a.verify:
        import layout
        from oracle import fv as ofv, grid as og, poisson, simple, krylov
        G = og.Grid(n, n, n, a.map)
        T = poisson.TPF(G)
        W = ofv.pack(ofv.weights(G))
        lid = ofv.lid_velocity(alpha)
        for key, Ud in states.items():
            if isinstance(key, tuple):
                continue
            Uo = layout.to_oracle(Ud.cpu().numpy(), (n, n, n))
            r = krylov.steady_residual(G, T, Uo, key, lid)[3]
            res["verify"][f"steady_residual_re{key:g}"] = float(r)
            ev = states.get(("evec", key))
            if ev is not None:
                e, lam0 = ev
                e = e.cpu().numpy()
                x = layout.to_oracle(e[:g.n_vel], (n, n, n)), layout.to_oracle(e[g.n_vel:], (n, n, n))
                Ar = ofv.pack(simple.krylov_vector(G, T, Uo, x[0], key)[0])
                Ai = ofv.pack(simple.krylov_vector(G, T, Uo, x[1], key)[0])
                z = ofv.pack(x[0]) + 1j * ofv.pack(x[1])
                rr = np.sqrt(np.sum(W * np.abs(Ar + 1j * Ai - lam0 * z) ** 2))
                res["verify"][f"eigen_residual_rel_re{key:g}"] = float(rr / abs(lam0))
        print(json.dumps(res["verify"]), flush=True)
    json.dump(res, open(a.out, "w"), indent=1)


if __name__ == "__main__":
    main()
