"""Wire model and dense retarded Green's function, FP64 (oracle; test infrastructure only).

Model (Sec. III.A and the lead/scattering self-energies of Sec. II.A):

* Sites of a W x L square lattice, slice-major: site (k, a) -> index k*W + a, slice k = 0..L-1
  along the wire, a = 0..W-1 across it.  H has the onsite energies on its diagonal and -t between
  nearest neighbours, along and across the slices.
* Buttiker scattering is diagonal in the site basis with sigma_i = -i*gamma_i/2 (Sec. III.A,
  Eq. for sigma_i; Sec. II.F, Eq. buttiker_scattering_gamma).  gamma_i is called ``eta`` here.
* Two leads: L couples to slice 0 and R to slice L-1.  lead_model 0 (default) is an exact clean
  semi-infinite square-lattice strip of the same width (onsite 0, hopping -t).  It is diagonal
  in the transverse sine modes phi_m with eigen-self-energies Sigma_m = t^2 g_s(E - eps_m), where
  g_s is the surface Green's function of a semi-infinite chain.  lead_model 1 is the paper's
  wide-band model Sigma_p = -(i/2) Gamma_l P_p (Sec. III.A), which has the same eigenvectors.
* G^r = (E - H - Sigma_L - Sigma_R - Sigma_s)^{-1}   (Eq. eq_for_gr), by dense LU.
* Multi-orbital slices (the "more orbitals per atom" generalisation of the Hamiltonian, Sec.
  "Generalizations of the Hamiltonian", and the s and p orbitals of the paper's tight-binding
  model, Sec. III.A): ``slice_h`` [W, W] real symmetric replaces the square-lattice
  cross-section: H_kk = slice_h + diag(onsite_k), W now counting orbitals (atoms x orbitals per
  atom).  The coupling between slices stays -t between the same orbital of neighbouring slices
  (orbital-diagonal).  The exact lead is then the clean strip of slice_h: its modes are the
  eigenvectors of slice_h (numpy eigh, a library step), eps their eigenvalues, and
  Sigma_m = t^2 g_s(E - eps_m) as before.
"""
import numpy as np


def hamiltonian(onsite, t, slice_h=None):
    """Dense real-symmetric tight-binding H for an [L, W] array of onsite energies (with
    ``slice_h``: the multi-orbital slice block on every slice, plus the onsite energies)."""
    onsite = np.asarray(onsite, dtype=np.float64)
    L, W = onsite.shape
    n = L * W
    H = np.zeros((n, n), dtype=np.float64)
    for k in range(L):
        if slice_h is not None:
            H[k * W:(k + 1) * W, k * W:(k + 1) * W] = np.asarray(slice_h, dtype=np.float64)
        for a in range(W):
            i = k * W + a
            H[i, i] += onsite[k, a]
            if slice_h is None and a + 1 < W:
                H[i, i + 1] = H[i + 1, i] = -t
            if k + 1 < L:
                H[i, i + W] = H[i + W, i] = -t
    return H


def transverse_modes(W, t, slice_h=None):
    """Modes of a W-site cross-section: the sine modes of the hopping -t chain (phi[a, m],
    eps[m], m = 1..W), or with ``slice_h`` its eigenvectors and eigenvalues (ascending)."""
    if slice_h is not None:
        eps, phi = np.linalg.eigh(np.asarray(slice_h, dtype=np.float64))
        return phi, eps
    a = np.arange(1, W + 1, dtype=np.float64)[:, None]
    m = np.arange(1, W + 1, dtype=np.float64)[None, :]
    phi = np.sqrt(2.0 / (W + 1)) * np.sin(m * np.pi * a / (W + 1))
    eps = -2.0 * t * np.cos(np.arange(1, W + 1) * np.pi / (W + 1))
    return phi, eps


def chain_surface_self_energy(e, t):
    """t^2 g_s(e) for a semi-infinite chain (onsite 0, hopping -t), retarded branch.

    g_s solves t^2 g^2 - e g + 1 = 0; inside the band |e| < 2t the root with Im g < 0 is the
    retarded one, outside it the root with |g| < 1/t (decaying).  Returns (Sigma, Gamma) with
    Gamma = i(Sigma - Sigma^*) = -2 Im Sigma (Eq. gamma_p_defined).
    """
    e = float(e)
    if abs(e) < 2.0 * t:
        s = 0.5 * (e - 1j * np.sqrt(4.0 * t * t - e * e))
    else:
        s = 0.5 * (e - np.sign(e) * np.sqrt(e * e - 4.0 * t * t)) + 0j
    return s, -2.0 * s.imag


def lead_modes(E, W, t, lead_model=0, gamma_lead=0.0, slice_h=None):
    """Eigen-decomposition of one lead's self-energy on its boundary slice.

    Returns phi [W, W] (columns = eigenvectors |i> of Gamma_p, Sec. II.D Step 3), sigma [W]
    complex eigenvalues of Sigma_p and gam [W] real eigenvalues of Gamma_p (lambda_i).
    """
    phi, eps = transverse_modes(W, t, slice_h)
    if lead_model == 0:
        sig = np.empty(W, dtype=np.complex128)
        gam = np.empty(W, dtype=np.float64)
        for m in range(W):
            sig[m], gam[m] = chain_surface_self_energy(E - eps[m], t)
    elif lead_model == 1:
        sig = np.full(W, -0.5j * gamma_lead, dtype=np.complex128)
        gam = np.full(W, float(gamma_lead))
    else:
        raise ValueError("lead_model must be 0 or 1")
    return phi, sig, gam


def lead_matrices(E, L, W, t, lead_model=0, gamma_lead=0.0, slice_h=None):
    """Sigma_L, Sigma_R, Gamma_L, Gamma_R embedded as dense n x n matrices (Eq. sigmas_comp_r)."""
    n = L * W
    phi, sig, gam = lead_modes(E, W, t, lead_model, gamma_lead, slice_h)
    s_blk = phi @ np.diag(sig) @ phi.T
    g_blk = phi @ np.diag(gam) @ phi.T
    out = []
    for k in (0, L - 1):
        S = np.zeros((n, n), dtype=np.complex128)
        Gm = np.zeros((n, n), dtype=np.complex128)
        S[k * W:(k + 1) * W, k * W:(k + 1) * W] += s_blk
        Gm[k * W:(k + 1) * W, k * W:(k + 1) * W] += g_blk
        out.append((S, Gm))
    (SL, GL), (SR, GR) = out
    return SL, SR, GL, GR


def green_retarded(E, onsite, eta, t, lead_model=0, gamma_lead=0.0, slice_h=None):
    """Dense G^r(E) = (E - H - Sigma^r)^{-1} (Eq. eq_for_gr) with
    Sigma^r = Sigma_L + Sigma_R + Sigma_s (Eq. sigmas_comp_r), Sigma_s = -i eta/2 per site.

    Returns a dict with G, H, the embedded lead matrices and gamma (= eta flattened).
    Pinned by: 2-site closed-form inverse, clean-chain transmission 1 in band / 0 outside,
    channel staircase of a clean strip, symmetry G = G^T and the sum rule A = G Gamma G^dag.
    """
    onsite = np.asarray(onsite, dtype=np.float64)
    eta = np.asarray(eta, dtype=np.float64)
    L, W = onsite.shape
    n = L * W
    H = hamiltonian(onsite, t, slice_h)
    SL, SR, GL, GR = lead_matrices(E, L, W, t, lead_model, gamma_lead, slice_h)
    gamma = eta.reshape(n)
    Ss = np.diag(-0.5j * gamma)
    M = E * np.eye(n) - H - SL - SR - Ss
    G = np.linalg.solve(M, np.eye(n, dtype=np.complex128))
    return dict(G=G, H=H, SigL=SL, SigR=SR, GamL=GL, GamR=GR, gamma=gamma, L=L, W=W, n=n)
