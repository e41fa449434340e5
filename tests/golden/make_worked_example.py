"""Writes worked_example_L2_K2.json: a hand-checkable EM iteration.

With L = 2 and K = 2 each observation is one pixel (l = 1) and the template of
shift s = (s1, s2) is P R_s x = x[(-s1) mod 2, (-s2) mod 2] = x[s1, s2].  EM for
SR-MRA then reduces to EM for a four-component 1-D Gaussian mixture whose means are
the four pixels and whose mixing weights are rho1[s1] * rho2[s2] (Sec. 2, Eqs.
weights_EM, x_EM, rho_EM; reading R2 for the product form of rho).  The expected
values below are that closed form, evaluated with the standard library only; no
oracle and no CUDA code is involved.
"""
import json
import math
import os

x = [[0.0, 1.0], [2.0, 3.0]]
y = [0.0, 1.0, 2.5]
sigma = 0.5
rho1 = [0.25, 0.75]
rho2 = [0.6, 0.4]

shifts = [(0, 0), (0, 1), (1, 0), (1, 1)]
w = []
lse = []
for yi in y:
    terms = [rho1[a] * rho2[b] * math.exp(-((yi - x[a][b]) ** 2) / (2 * sigma * sigma))
             for a, b in shifts]
    tot = sum(terms)
    lse.append(math.log(tot))
    w.append([t / tot for t in terms])
N = len(y)
x_new = [[0.0, 0.0], [0.0, 0.0]]
for k, (a, b) in enumerate(shifts):
    num = sum(w[i][k] * y[i] for i in range(N))
    den = sum(w[i][k] for i in range(N))
    x_new[a][b] = num / den
joint = [sum(w[i][k] for i in range(N)) / N for k in range(4)]
rho1_new = [joint[0] + joint[1], joint[2] + joint[3]]
rho2_new = [joint[0] + joint[2], joint[1] + joint[3]]

out = dict(
    description="L=2, K=2, N=3 worked example: SR-MRA EM reduces to a 4-component "
                "Gaussian mixture EM; expected values are its closed form.",
    L=2, K=2, sigma=sigma, x=x, y=y, rho1=rho1, rho2=rho2,
    expected=dict(weights=w, lse=lse, loglik=sum(lse), x=x_new,
                  rho1=rho1_new, rho2=rho2_new))
path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "worked_example_L2_K2.json")
with open(path, "w") as f:
    json.dump(out, f, indent=1)
print("wrote", path)
