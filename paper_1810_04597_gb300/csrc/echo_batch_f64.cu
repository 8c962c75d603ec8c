// echo_batch_f64.cu -- batched-run kernels for double storage.
#include "echo_batch_kernels.cuh"

namespace echo {

template <>
const void *batch_stage_kernel<double>(int mk, bool mlp)
{
    if (mk == 1)
        return mlp ? (const void *)k_batch_stage<1, double, 3, 4> : (const void *)k_batch_stage<1, double, 0, 4>;
    return mlp ? (const void *)k_batch_stage<0, double, 3, 4> : (const void *)k_batch_stage<0, double, 0, 4>;
}

template <int MK>
static void guess_pass(const RunDesc<double> *descs, const BatchPlan *planp, const BatchPlan &P, float gr_f, cudaStream_t s)
{
    // the grid is sized for the whole GPU: the lists' lengths are on the device
    static int resident = 0;
    if (resident == 0)
        resident = tc_resident_ctas((const void *)k_bphase_guess_tc<MK, double>, TC_SMEM);
    k_bphase_guess_tc<MK, double><<<(unsigned)resident, 128, TC_SMEM, s>>>(descs, planp, gr_f);
    k_bphase_clear_lists<double><<<1, 32, 0, s>>>(descs, P.nruns);
}

template <>
void batch_enqueue_guess<double>(int mk, const void *descs, const BatchPlan *plan_dev, const BatchPlan &plan, float gr_f,
                            cudaStream_t s)
{
    const RunDesc<double> *d = static_cast<const RunDesc<double> *>(descs);
    if (mk == 1)
        guess_pass<1>(d, plan_dev, plan, gr_f, s);
    else
        guess_pass<0>(d, plan_dev, plan, gr_f, s);
}

template <int MK>
static void phased(bool mlp, const RunDesc<double> *descs, const BatchPlan *planp, const BatchPlan &P, int nruns,
                   const Phys &ph, int guess, double dt, double cfl, cudaStream_t s)
{
    k_bphase_scalars<double><<<1, 32, 0, s>>>(descs, nruns, 0, dt, cfl);
    for (int st = 0; st < 3; ++st) {
        for (int p = PH_FILLF0; p <= PH_FILLF2; ++p)
            k_bphase_fill<double><<<(unsigned)P.ntiles[p], 128, 0, s>>>(descs, planp, p);
        if (mlp) {
            guess_pass<MK>(descs, planp, P, ph.gr_f, s);
            k_bphase_c2p<MK, double, 3><<<(unsigned)P.ntiles[PH_C2P], 128, 0, s>>>(descs, planp, ph, guess, st == 0 ? 1 : 0);
        } else {
            k_bphase_c2p<MK, double, 0><<<(unsigned)P.ntiles[PH_C2P], 128, 0, s>>>(descs, planp, ph, guess, st == 0 ? 1 : 0);
        }
        if (st == 0)
            k_bphase_scalars<double><<<1, 32, 0, s>>>(descs, nruns, 1, dt, cfl);
        for (int p = PH_FILLP0; p <= PH_FILLP2; ++p)
            k_bphase_fill<double><<<(unsigned)P.ntiles[p], 128, 0, s>>>(descs, planp, p);
        k_bphase_faces<MK, double><<<(unsigned)P.ntiles[PH_FACES], 128, 0, s>>>(descs, planp, ph);
        k_bphase_emf<MK, double><<<(unsigned)P.ntiles[PH_EMF], 128, 0, s>>>(descs, planp);
        k_bphase_update<MK, double><<<(unsigned)P.ntiles[PH_UPDATE], 128, 0, s>>>(descs, planp, ph, st);
    }
}

template <>
void batch_enqueue_phased<double>(int mk, bool mlp, const void *descs, const BatchPlan *plan_dev, const BatchPlan &plan,
                              int nruns, const Phys &ph, int guess, double dt, double cfl, cudaStream_t s)
{
    const RunDesc<double> *d = static_cast<const RunDesc<double> *>(descs);
    if (mk == 1)
        phased<1>(mlp, d, plan_dev, plan, nruns, ph, guess, dt, cfl, s);
    else
        phased<0>(mlp, d, plan_dev, plan, nruns, ph, guess, dt, cfl, s);
}

}  // namespace echo
