"""Seeded synthetic inputs shaped like the paper's workloads.

This module only builds target parameters and starting points (numpy, its own
PCG64 streams).  It contains none of the sampling arithmetic: the CUDA path and
the CPU oracle both receive the arrays it returns.

Workloads (all synthetic; the paper's UCI / PosteriorDB data is not used):
  * gauss_conj  -- ESS on a conjugate Gaussian: prior N(0, Sigma), Sigma = A A^T/16 + I,
                   A ~ N(0,1) (d x d); one observation y ~ N(x_true, 0.5^2 I) with
                   x_true ~ N(0, Sigma).  Closed-form posterior (Sec. 7.2 stand-in).
  * gp_logit    -- ESS on latent GP classification: d inputs ~ U[0,1], RBF kernel with
                   length-scale 0.1 plus 1e-6 jitter, Cholesky in FP64 stored in FP32,
                   labels ~ Bernoulli(sigmoid(f_true)), f_true = L z (Fig. 1 / Sec. 7.2
                   stand-in: a GP posterior with an expensive O(d^2) prior draw).
  * funnel      -- Neal's funnel, v ~ N(0, 3^2), x_i | v ~ N(0, e^v) (no data).
  * logreg      -- Bayesian logistic regression: X (n x d) ~ N(0,1) stored in FP32,
                   beta ~ N(0,1), y ~ Bernoulli(sigmoid(X beta)) (Sec. 7.3/7.4 stand-in).
  * gauss_diag  -- N(mu, diag(sigma^2)) used by the NUTS and DR moment tests.
"""
import numpy as np

DATA_SEED = 0x2503_17405
CHAIN_SEED = 1


def _rng(seed, stream):
    return np.random.default_rng([seed, stream])


def gauss_conj(d=16, seed=DATA_SEED, noise_sd=0.5):
    r = _rng(seed, 1)
    A = r.standard_normal((d, d))
    Sigma = A @ A.T / 16.0 + np.eye(d)
    L = np.linalg.cholesky(Sigma)
    x_true = L @ r.standard_normal(d)
    y = x_true + noise_sd * r.standard_normal(d)
    s2 = noise_sd ** 2
    params = np.concatenate([L.ravel(), y, [s2]])
    # closed-form posterior of x given y (Gaussian prior x Gaussian likelihood)
    prec = np.linalg.inv(Sigma) + np.eye(d) / s2
    post_cov = np.linalg.inv(prec)
    post_mean = post_cov @ (y / s2)
    return dict(kind="gauss_conj", d=d, n_data=0, params=params, L=L, y=y, s2=s2,
                Sigma=Sigma, post_mean=post_mean, post_cov=post_cov)


def gp_logit(d=256, seed=DATA_SEED, lengthscale=0.1, jitter=1e-6):
    r = _rng(seed, 2)
    u = r.uniform(0.0, 1.0, d)
    K = np.exp(-(u[:, None] - u[None, :]) ** 2 / (2.0 * lengthscale ** 2)) + jitter * np.eye(d)
    L = np.linalg.cholesky(K).astype(np.float32).astype(np.float64)  # FP64 factor, FP32 storage
    f_true = L @ r.standard_normal(d)
    labels = (r.uniform(0.0, 1.0, d) < 1.0 / (1.0 + np.exp(-f_true))).astype(np.float64)
    s = 2.0 * labels - 1.0
    params = np.concatenate([L.ravel(), s])
    return dict(kind="gp_logit", d=d, n_data=0, params=params, L=L, s=s, inputs=u)


def funnel(d=10):
    return dict(kind="funnel", d=d, n_data=0, params=np.zeros(0))


def logreg(n=1000, d=25, seed=DATA_SEED):
    r = _rng(seed, 3)
    X = r.standard_normal((n, d)).astype(np.float32).astype(np.float64)
    beta = r.standard_normal(d)
    p = 1.0 / (1.0 + np.exp(-(X @ beta)))
    y = (r.uniform(0.0, 1.0, n) < p).astype(np.float64)
    params = np.concatenate([X.ravel(), y])
    return dict(kind="logreg", d=d, n_data=n, params=params, X=X, y=y, beta_true=beta)


def gauss_diag(d=8, seed=DATA_SEED):
    r = _rng(seed, 4)
    mu = r.standard_normal(d)
    sd = np.exp(r.uniform(-0.5, 0.5, d))
    return dict(kind="gauss_diag", d=d, n_data=0, params=np.concatenate([mu, sd]), mu=mu, sd=sd)


def std_normal(d=1):
    """N(0, I_d) as a diagonal Gaussian (the target of the paper's delayed-rejection toy)."""
    mu, sd = np.zeros(d), np.ones(d)
    return dict(kind="gauss_diag", d=d, n_data=0, params=np.concatenate([mu, sd]), mu=mu, sd=sd)


def mog(d=100, rho=0.99, offsets=(-10.0, 0.0, 10.0), weights=None):
    """Sec. 7.3's NUTS target: an equal-weight mixture of Gaussians with unit variances and
    correlation rho between every pair of coordinates, the modes on the principal direction at
    offset * (1, ..., 1).  params = rho, w[K], mu[K * d] with n_data = K."""
    K = len(offsets)
    w = np.ones(K) if weights is None else np.asarray(weights, dtype=np.float64)
    mu = np.outer(np.asarray(offsets, dtype=np.float64), np.ones(d))
    return dict(kind="mog", d=d, n_data=K, params=np.concatenate([[rho], w, mu.ravel()]),
                rho=rho, w=w, mu=mu)


def x0_mog_exact(w, m, seed=DATA_SEED, stream=15):
    """Exact draws: a component by weight, then mu_k + sqrt(1 - rho) z + sqrt(rho) zeta 1
    (covariance (1 - rho) I + rho 1 1^T; rho >= 0)."""
    r = _rng(seed, stream)
    k = r.choice(len(w["w"]), size=m, p=w["w"] / w["w"].sum())
    z = r.standard_normal((m, w["d"]))
    zeta = r.standard_normal((m, 1))
    return w["mu"][k] + np.sqrt(1.0 - w["rho"]) * z + np.sqrt(w["rho"]) * zeta


def gp_reg(n=100, p=6, seed=DATA_SEED, theta_true=(0.3, 1.0, 0.4)):
    """Sec. 7.2's GP-regression hyperparameter posterior on synthetic data shaped like its
    house-price task: n points with p = 6 standardised features, y drawn from the model at
    theta_true = (sigma, tau, lambda) and standardised.  ESS target over x = (sigma, tau, lambda)
    with the N(0, I_3) prior (L = I_3); params = L[9], D[n*n] (squared distances), y[n]."""
    r = _rng(seed, 7)
    X = r.standard_normal((n, p))
    X = (X - X.mean(0)) / X.std(0)
    D = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    s, t, l = theta_true
    C = t * t * np.exp(-l * l * D) + s * s * np.eye(n)
    y = np.linalg.cholesky(C) @ r.standard_normal(n)
    y = (y - y.mean()) / y.std()
    L = np.eye(3)
    return dict(kind="gp_reg", d=3, n_data=n, params=np.concatenate([L.ravel(), D.ravel(), y]),
                X=X, D=D, y=y, theta_true=np.array(theta_true))


def x0_gp_reg(w, m, seed=DATA_SEED, stream=16):
    """Starts near the data-generating hyperparameters: theta_true + 0.05 z."""
    return w["theta_true"][None, :] + 0.05 * _rng(seed, stream).standard_normal((m, 3))


def flat(d=8, seed=DATA_SEED):
    r = _rng(seed, 5)
    A = r.standard_normal((d, d))
    L = np.linalg.cholesky(A @ A.T / d + np.eye(d))
    return dict(kind="flat", d=d, n_data=0, params=L.ravel(), L=L)


# ---- starting points ------------------------------------------------------------
def x0_zeros(m, d):
    return np.zeros((m, d))


def x0_normal(m, d, seed=DATA_SEED, scale=1.0, stream=10):
    return scale * _rng(seed, stream).standard_normal((m, d))


def x0_gauss_posterior(w, m, seed=DATA_SEED, stream=11):
    """Exact draws from the conjugate-Gaussian posterior (exact-start chains)."""
    C = np.linalg.cholesky(w["post_cov"])
    z = _rng(seed, stream).standard_normal((m, w["d"]))
    return w["post_mean"][None, :] + z @ C.T


def x0_funnel_exact(m, d=10, seed=DATA_SEED, stream=12):
    """Exact draws from the funnel by ancestral sampling (exact-start chains)."""
    r = _rng(seed, stream)
    v = 3.0 * r.standard_normal(m)
    x = r.standard_normal((m, d - 1)) * np.exp(v / 2.0)[:, None]
    return np.concatenate([v[:, None], x], axis=1)


def x0_gauss_diag_exact(w, m, seed=DATA_SEED, stream=13):
    z = _rng(seed, stream).standard_normal((m, w["d"]))
    return w["mu"][None, :] + z * w["sd"][None, :]


def x0_logreg(w, m, seed=DATA_SEED, stream=14):
    """Chains start near the posterior mode region: beta_true + 0.05 N(0,1) jitter.

    The paper does not state x0; beta0 = 0 would put the first draws far out in
    the tails, so a small jitter around the data-generating beta is used.
    """
    z = _rng(seed, stream).standard_normal((m, w["d"]))
    return w["beta_true"][None, :] + 0.05 * z


# ---- serving stream (Poisson arrivals) --------------------------------------------
def serving_jobs(n_jobs=200, seed=DATA_SEED, rate_hz=50.0, scale=1.0):
    """Mixed request stream: ESS-GP (d ~ logU[64,1024]) and NUTS-logistic
    (d ~ logU[10,100], n ~ logU[1e3,1e4]) 50/50; chains ~ logU[16,4096];
    draws ~ logU[500,5000]; exponential inter-arrival times at rate_hz.
    `scale` < 1 shrinks chains and draws (for tests)."""
    r = _rng(seed, 20)

    def logu(a, b):
        return float(np.exp(r.uniform(np.log(a), np.log(b))))

    t = 0.0
    jobs = []
    for k in range(n_jobs):
        t += r.exponential(1.0 / rate_hz)
        kind = "ess_gp" if r.uniform() < 0.5 else "nuts_logreg"
        chains = max(1, int(round(logu(16, 4096) * scale)))
        draws = max(2, int(round(logu(500, 5000) * scale)))
        if kind == "ess_gp":
            d = int(round(logu(64, 1024)))
            jobs.append(dict(id=k, arrival=t, kind=kind, d=d, n_data=0, chains=chains,
                             draws=draws, data_seed=int(r.integers(1 << 31))))
        else:
            d = int(round(logu(10, 100)))
            n = int(round(logu(1e3, 1e4)))
            jobs.append(dict(id=k, arrival=t, kind=kind, d=d, n_data=n, chains=chains,
                             draws=draws, data_seed=int(r.integers(1 << 31))))
    return jobs
