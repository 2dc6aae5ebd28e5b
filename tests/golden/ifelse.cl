__kernel void sel(__global int *data)
{
    if (16u > get_local_id(0)) {
        data[get_local_id(0)] = 7;
    } else {
        data[get_local_id(0)] = 9;
    }
}
