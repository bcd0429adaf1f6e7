"""Write FP64 oracle histories used as stored expected values by the GPU tests.

Calls only the oracle (and the shared seeded input generator).  Each output
file starts with a header naming the case and this command.

  python tests/golden/make_oracle_histories.py lbe256      # ~10 min on 8 cores
  python tests/golden/make_oracle_histories.py c2 lbe      # 128^3, 2000 steps
  python tests/golden/make_oracle_histories.py c2 dugks    # 128^3, 2000 steps (~1.5 h)
  python tests/golden/make_oracle_histories.py c3 lbe      # 64^3, 1000 steps
  python tests/golden/make_oracle_histories.py c3 dugks    # 64^3, 1000 steps
  python tests/golden/make_oracle_histories.py f3 lbe 52.12     # 64^3, 400 time units
  python tests/golden/make_oracle_histories.py f3 dugks 104.24  # 64^3, 800 steps (~5 min)

Cases
  lbe256  256^3, k0 = 8, Ma = 0.15, Re_lambda = 70, seed 1300: MRT-LBE E and
          eps every 5 steps until the state is non-finite (the 256^3 timing
          field, whose LBE run blows up; Sec. IV.E discusses LBE stability).
  c2      128^3, k0 = 8, Ma = 0.1, Re_lambda = 25, seed 1200, 2000 steps of
          the named scheme (DUGKS dt = 0.5): E and eps every 10 steps, E(k)
          every 200 steps.
  c3      64^3 version of the 256^3 timing field: k0 = 8, Ma = 0.15,
          Re_lambda = 70, seed 1300, 1000 steps (DUGKS dt = 0.5), E and eps
          every 10 steps, E(k) every 200 steps, until non-finite.
  f3      64^3 box of the Sec. IV.D decay workload: spectrum shape
          k^4 exp(-0.14 k^2) (k0 = sqrt(2/0.14)), u' = 0.032 (Ma = u'/c_s),
          seed 1700, nu from the named Re_lambda (52.12 or 104.24); 400
          lattice time units (MRT-LBE dt = 1, DUGKS dt = 0.5), E and eps
          every 10 time units.
"""
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import kin_inputs as ki  # noqa: E402
import oracle  # noqa: E402


def lbe256():
    N, seed, k0, Ma, re = 256, 1300, 8.0, 0.15, 70.0
    u, info = ki.dhit_velocity(N, seed, k0, Ma, return_info=True)
    nu = ki.nu_from_re_lambda(info["u_prime"], info["omega"], re)
    f = oracle.equilibrium_field(u)
    del u
    path = os.path.join(HERE, "oracle_lbe_256_blowup.txt")
    with open(path, "w") as fh:
        fh.write("# FP64 oracle, MRT-LBE, 256^3, k0=%g Ma=%g Re_lambda=%g seed=%d nu=%.17g\n"
                 % (k0, Ma, re, seed, nu))
        fh.write("# written by: python tests/golden/make_oracle_histories.py lbe256\n")
        fh.write("# step E eps\n")
        E, eps = oracle.stats(f, nu)
        fh.write("0 %.17g %.17g\n" % (E, eps))
        for n in range(1, 201):
            f = oracle.lbe_step(f, nu)
            if n % 5 == 0:
                E, eps = oracle.stats(f, nu)
                if not (math.isfinite(E) and math.isfinite(eps)) or E > 1e300:
                    fh.write("%d nonfinite nonfinite\n" % n)
                    break
                fh.write("%d %.17g %.17g\n" % (n, E, eps))
                fh.flush()


def c2(scheme, case="c2", N=128, seed=1200, k0=8.0, Ma=0.1, re=25.0, steps=2000):
    dt = 1.0 if scheme == "lbe" else 0.5
    u, info = ki.dhit_velocity(N, seed, k0, Ma, return_info=True)
    nu = ki.nu_from_re_lambda(info["u_prime"], info["omega"], re)
    f = oracle.equilibrium_field(u)
    del u
    nsh = 1 + int(math.floor(math.sqrt(3 * (N // 2) ** 2) + 0.5))
    hist = os.path.join(HERE, "oracle_%s_%d_%s.txt" % (case, N, scheme))
    spec = os.path.join(HERE, "oracle_%s_%d_%s_spectrum.txt" % (case, N, scheme))
    t0 = time.time()
    with open(hist, "w") as fh, open(spec, "w") as fs:
        for h in (fh, fs):
            h.write("# FP64 oracle, %s, %d^3, k0=%g Ma=%g Re_lambda=%g seed=%d nu=%.17g dt=%g\n"
                    % (scheme, N, k0, Ma, re, seed, nu, dt))
            h.write("# written by: python tests/golden/make_oracle_histories.py %s %s\n" % (case, scheme))
        fh.write("# step E eps\n")
        fs.write("# step E(s) for s = 0..%d\n" % (nsh - 1))
        for n in range(steps + 1):
            if n % 10 == 0:
                _, uu = oracle.macro(f)
                E, eps = oracle.energy_dissipation(uu, nu)
                if not (math.isfinite(E) and math.isfinite(eps)):
                    fh.write("%d nonfinite nonfinite\n" % n)
                    break
                fh.write("%d %.17g %.17g\n" % (n, E, eps))
                fh.flush()
                if n % 200 == 0:
                    Ek, _ = oracle.spectrum(uu, nsh)
                    fs.write("%d %s\n" % (n, " ".join("%.17g" % v for v in Ek)))
                    fs.flush()
            if n < steps:
                f = oracle.step(scheme, f, nu, dt)
            if n % 100 == 0:
                print(scheme, n, "%.0f s" % (time.time() - t0), flush=True)


def f3(scheme, re, N=64, seed=1700, T=400, every=10):
    k0, Ma = math.sqrt(2.0 / 0.14), 0.032 / math.sqrt(1.0 / 3.0)
    dt = 1.0 if scheme == "lbe" else 0.5
    per = int(round(1.0 / dt))
    u, info = ki.dhit_velocity(N, seed, k0, Ma, return_info=True)
    nu = ki.nu_from_re_lambda(info["u_prime"], info["omega"], re)
    f = oracle.equilibrium_field(u)
    del u
    path = os.path.join(HERE, "oracle_f3_%d_%s_re%g.txt" % (N, scheme, re))
    t0 = time.time()
    with open(path, "w") as fh:
        fh.write("# FP64 oracle, %s, %d^3, k0=%.17g Ma=%.17g Re_lambda=%g seed=%d nu=%.17g dt=%g\n"
                 % (scheme, N, k0, Ma, re, seed, nu, dt))
        fh.write("# written by: python tests/golden/make_oracle_histories.py f3 %s %g\n" % (scheme, re))
        fh.write("# time E eps\n")
        for t in range(0, T + 1, every):
            E, eps = oracle.stats(f, nu)
            fh.write("%d %.17g %.17g\n" % (t, E, eps))
            fh.flush()
            if t < T:
                for _ in range(every * per):
                    f = oracle.step(scheme, f, nu, dt)
            print(scheme, re, t, "%.0f s" % (time.time() - t0), flush=True)


if __name__ == "__main__":
    if sys.argv[1] == "lbe256":
        lbe256()
    elif sys.argv[1] == "c2":
        c2(sys.argv[2])
    elif sys.argv[1] == "f3":
        f3(sys.argv[2], float(sys.argv[3]))
    elif sys.argv[1] == "c3":
        c2(sys.argv[2], case="c3", N=64, seed=1300, k0=8.0, Ma=0.15, re=70.0, steps=1000)
    else:
        raise SystemExit(__doc__)
